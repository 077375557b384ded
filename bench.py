"""Benchmark of the DMD hot path on the 128^3 x 3 workload (one JSON line).

One step = the whole hot path on one synthetic snapshot matrix: dmd_fit
(rSVD at r = 150, oversample 10, 2 power iterations, modes, amplitudes) of the
n = 6,291,456 x 201 FP32 snapshots, then dmd_predict of 1000 frames (k = 0..999)
written as FP32.  `value` is frames per second of whole steps (1000 frames per
step over fit + reconstruction); the fit seconds and the reconstruction-only
frames/s are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32]
                  [--impl ours|reference] [--config cfg1|cfg0]

Under torchrun each rank runs an independent replica on its own GPU (the fit
has no cross-rank exchange in this build): value = all ranks' frames / the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on a
bounded row sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "DMD fit s & recon frames/s, 128³ r=150: mixed vs FP32 on GB300 at rel err≤1e-4"
CONFIGS = {
    # name: (grid N, dim, m, r, oversample, power_iters, frames)
    "cfg1": dict(N=128, dim=3, m=200, r=150, oversample=10, power_iters=2, frames=1000, seed=1001,
                 workload="3D 128^3 x 3 velocity (n=6,291,456), m=200 FP32 snapshots, 150 modes + quadratic "
                          "term 1e-3 + noise 1e-4; rSVD r=150 p=10 q=2; reconstruct k=0..999"),
    "cfg0": dict(N=64, dim=2, m=100, r=20, oversample=10, power_iters=2, frames=501, seed=1000,
                 workload="2D 64^2 x 2 velocity (n=8192), m=100, 20 modes, noise 1e-8; r=20; predict k=0..500"),
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def make_scene(cfg, device):
    from paper_2502_05339_gb300 import synth
    c = CONFIGS[cfg]
    if cfg == "cfg1":
        return synth.config1(seed=c["seed"], device=device)
    return synth.config0(seed=c["seed"], device=device)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    from paper_2502_05339_gb300 import dmd
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    c = CONFIGS[args.config]
    prec = args.precision
    sc = make_scene(args.config, dev)
    torch.cuda.synchronize()
    n, m, r, K = sc.n, sc.m, c["r"], c["frames"]
    S = sc.S
    ks = torch.arange(K, dtype=torch.int32, device=dev)
    out = torch.empty((K, dmd.round_up(n, 32)), dtype=torch.float32, device=dev)
    L = dmd.lib()
    st = torch.cuda.current_stream(dev)

    def step():
        model = dmd.dmd_fit(S, n, r, oversample=c["oversample"], power_iters=c["power_iters"],
                            precision=prec, seed=c["seed"])
        dmd.dmd_predict(model, ks, precision=prec, out=out)
        return model

    for _ in range(args.warmup):
        model = step()
    torch.cuda.synchronize()
    model.check()
    # fit-only and reconstruction-only timings (events on the launching stream)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    fit_ms, rec_ms = [], []
    for _ in range(max(1, min(3, args.steps))):
        e0.record(st)
        model = dmd.dmd_fit(S, n, r, oversample=c["oversample"], power_iters=c["power_iters"], precision=prec,
                            seed=c["seed"])
        e1.record(st)
        dmd.dmd_predict(model, ks, precision=prec, out=out)
        e2.record(st)
        torch.cuda.synchronize()
        fit_ms.append(e0.elapsed_time(e1))
        rec_ms.append(e1.elapsed_time(e2))
    model.check()
    fit_s = float(np.median(fit_ms)) / 1e3
    rec_s = float(np.median(rec_ms)) / 1e3

    # the timed region: exactly `steps` whole steps
    launches0 = L.dmd_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(st)
        for _ in range(args.steps):
            step()
        t1.record(st)
        torch.cuda.synchronize()
        barrier(world)
    elapsed = t0.elapsed_time(t1) / 1e3
    launches = (L.dmd_launch_count() - launches0) // max(args.steps, 1)
    elapsed_max = max_over_ranks(elapsed, world)
    frames_total = K * args.steps * world
    value = frames_total / elapsed_max

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = run_e2e(args, sc, c, dmd, dev, st, out, ks)

    peaks, peak_kind = load_peaks()
    clocks = clk.summary()
    roof = roofline(n, r, K, rec_s, prec, peaks, peak_kind)
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3" if prec == "mixed" else "f32",
        "data": "synthetic", "impl": "ours",
        "config": {"workload": c["workload"], "n": n, "m": m, "r": r, "frames": K, "precision": prec,
                   "parallelism": f"replicas{world}", "l2": "inputs (5.06 GB) and outputs (25.2 GB) exceed L2"},
        "fit_s": fit_s, "recon_frames_per_s": K / rec_s, "recon_s": rec_s,
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
        "parity": {"status": model.status()},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config, sample_rows=args.cpu_rows)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(args, sc, c, dmd, dev, st, out, ks):
    """Same step through the public API with HOST snapshots in and HOST frames out."""
    n, K = sc.n, c["frames"]
    try:
        S_host = torch.empty(sc.S.shape, dtype=torch.float32, pin_memory=True)
        S_host.copy_(sc.S.cpu())
        F_host = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
    except RuntimeError as e:
        return {"value": None, "unit": "frames/s", "error": f"pinned host buffers: {e}"}
    S_dev = torch.empty_like(sc.S)
    steps = max(1, min(args.steps, 3))

    def one():
        S_dev.copy_(S_host, non_blocking=True)
        model = dmd.dmd_fit(S_dev, n, c["r"], oversample=c["oversample"], power_iters=c["power_iters"],
                            precision=args.precision, seed=c["seed"])
        dmd.dmd_predict(model, ks, precision=args.precision, out=out)
        F_host.copy_(out, non_blocking=True)

    one()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        one()
    b.record(st)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    return {"value": K * steps / sec, "unit": "frames/s", "h2d_bytes_per_step": int(S_host.numel() * 4),
            "d2h_bytes_per_step": int(F_host.numel() * 4), "steps": steps}


def roofline(n, r, K, rec_s, prec, peaks, peak_kind):
    """Reconstruction launch F = Phi_R C (the largest single launch of a step)."""
    if prec == "mixed":
        bytes_ = 4.0 * n * (r + K)                 # read Phi_R once, write K frames
        achieved = bytes_ / rec_s / 1e9
        peak = float(peaks["hbm_gbs"])
        return {"kernel": "umma_nn (reconstruction)", "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None, "peak_source": peak_kind}
    flops = 2.0 * n * r * K
    achieved = flops / rec_s / 1e12
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12     # FP32 FFMA: 152 SMs x 128 lanes x 2 flops x clock
    return {"kernel": "k_gemm_nn_f32 (reconstruction)", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}


def cpu_baseline(cfg, sample_rows=None):
    """The FP64 oracle, as it stands, on a bounded row sample of the workload."""
    from oracle import dmd_oracle as O
    from paper_2502_05339_gb300 import synth
    c = CONFIGS[cfg]
    sc = make_scene(cfg, "cpu") if cfg == "cfg0" else None
    if cfg == "cfg1":
        # a 32^3 x 3 grid with the same recipe stands in for a row sample of 128^3 x 3
        N = 32
        sc = synth.linear_modes_scene(N, 3, 75, c["m"], c["seed"], sigma_lo=-0.02, noise=1e-4, nonlinear=1e-3)
    X = sc.X().numpy()
    t0 = time.perf_counter()
    ref = O.exact_dmd(X, c["r"])
    PhiR, beta, kinds = O.to_real_form(ref["Phi"], ref["lam"], ref["b"])
    t1 = time.perf_counter()
    ks = list(range(c["frames"]))
    O.predict_real(PhiR, O.coefficients(ref["lam"], beta, ks, kinds))
    t2 = time.perf_counter()
    n_full = 3 * 128 ** 3 if cfg == "cfg1" else sc.n
    scale = n_full / sc.n
    fit_s, pred_s = (t1 - t0) * scale, (t2 - t1) * scale
    cores = torch.get_num_threads()
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        pass
    return {"value": c["frames"] / (fit_s + pred_s), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{sc.name}: n={sc.n} rows ({sc.n / n_full:.4f} of the workload), m={c['m']}, r={c['r']}, "
                      f"{c['frames']} frames; times scaled by n (fit {fit_s:.1f} s, predict {pred_s:.1f} s "
                      f"at full n)",
            "measured_s": t2 - t0}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    c = CONFIGS[args.config]
    total = 0.0
    fr = 0
    base = None
    for _ in range(args.warmup):
        cpu_baseline(args.config)
    for _ in range(args.steps):
        base = cpu_baseline(args.config)
        total += base["measured_s"]
        fr += 1
    value = base["value"]
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / max(fr, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": c["workload"], "precision": "fp64 oracle"},
            "cpu_baseline": {k: base[k] for k in ("kind", "cores", "sample", "value", "unit")},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("DMD_BENCH_PRECISION", "fp32"), choices=["fp32", "mixed"])
    ap.add_argument("--config", default="cfg1", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=None)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
