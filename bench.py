"""Benchmark of the DMD hot path on the 128^3 x 3 workload (one JSON line).

One step = the whole hot path on one synthetic snapshot matrix: dmd_fit
(rSVD at r = 150, oversample 10, 2 power iterations, modes, amplitudes) of the
n = 6,291,456 x 201 FP32 snapshots, then dmd_predict of 1000 frames (k = 0..999)
written as FP32.  `value` is frames per second of whole steps (1000 frames per
step over fit + reconstruction) in the mixed (BF16x3 tensor-core) form by
default; the fit seconds and the reconstruction-only frames/s are reported
beside it, and `forms` gives the same three numbers for both the mixed and the
plain FP32 form side by side.  `kernels` holds a roofline entry per tall pass
of the step (each timed alone on the step's shapes); `roofline` is the entry
with the largest share of the step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32]
                  [--impl ours|reference] [--config cfg1|cfg0|...]
  python bench.py --case gram|tn|gramq|sketch|recon|loss|lossgrad|advect|optdmd [--rows N]

Under torchrun each rank runs an independent replica on its own GPU (the fit
has no cross-rank exchange in this build): value = all ranks' frames / the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on a
bounded row sample of the same workload on the host cores.
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
    "cfg2": dict(N=96, dim=3, m=300, r=100, q=8, oversample=10, power_iters=2, frames=1, rollout=200, seed=1002,
                 workload="DMDc 96^3 x 3 (n=2,654,208), m=300, q=8 Gaussian-blob forces, piecewise-constant "
                          "U(-1,1) inputs per 20 steps, 100 latent modes; fit r=100, roll out 200 steps, "
                          "adjoint of ||x_200 - x_target||^2 w.r.t. u_0..u_199 and b"),
    "cfg3": dict(N=0, dim=2, m=0, r=0, oversample=10, power_iters=2, frames=256, seed=1003, scenes=64,
                 workload="64 2D scenes, grid N log-uniform in [64, 512] (x2 components), m ~ U{50..400}, "
                          "r ~ U{10..128} (even), data as config 0 with noise 1e-5 and frequencies stratified over "
                          "(0, pi); each scene predicts 256 "
                          "frames; one batched call over 16 lanes"),
    "up": dict(N=128, dim=3, m=200, r=150, oversample=10, power_iters=2, frames=1000, seed=1001, coarse=32,
               threshold=0.3,
               workload="upsampling evolution (Sec. 6.3.1): the rank-150 model of the 128^3 x 3 scene, H_0 its "
                        "first snapshot, 1000 inputs from a 32^3 x 3 scene (75 pairs, other seed) prolonged x4 "
                        "to 128^3 x 3; modes with |Im log lambda| < 0.3 follow the inputs"),
    "adv": dict(N=128, dim=3, m=200, r=150, oversample=10, power_iters=2, frames=1000, seed=1001, dt=0.5,
                chunk=256,
                workload="density in the DMD velocity (Sec. 7.2): the rank-150 model of the 128^3 x 3 scene, "
                         "1000 semi-Lagrangian steps (dt 0.5 cells per unit velocity) of a cell-centred 128^3 "
                         "density (cosine pattern plus a Gaussian blob), velocity frames rebuilt 256 at a time"),
    "cfg4": dict(N=256, dim=3, m=300, r=150, oversample=16, power_iters=1, frames=2000, seed=1004,
                 workload="Large: 256^3 x 3 velocity (n=50,331,648), m=300 FP32 snapshots (60.6 GB), 150 modes + "
                          "quadratic term 1e-3 + noise 1e-4; rSVD r=150 p=16 q=1 (mixed), then 2000 frames "
                          "(k=0..1999) streamed into sum_k w_k ||x_k - x_tgt||^2 / 2 and its gradient w.r.t. "
                          "lambda and b, frames recomputed on the tensor cores and never stored"),
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
    """The slowest rank's time (all ranks get it)."""
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, elapsed_max: float, world: int) -> float:
    """Units all replicas processed over the slowest replica's time (weak scaling)."""
    return units_per_rank * world / elapsed_max


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
    value = whole_job_rate(K * args.steps, elapsed_max, world)

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = run_e2e(args, sc, c, dmd, dev, st, out, ks)
    adjoint = adjoint_timing(model, ks, out, dmd, st, prec, rec_s)
    optdmd = None if args.no_optdmd else optdmd_timing(S, n, c, dmd, st, prec, fit_s)

    peaks, peak_kind = load_peaks()
    clocks = clk.summary()
    kernels = [] if args.no_kernels else kernel_rooflines(sc, c, dmd, dev, st, prec, peaks, peak_kind)
    kernels.insert(0, roofline(n, r, K, rec_s, prec, peaks, peak_kind))
    for e in kernels:
        if TRAFFIC_PER_ROW.get(e["kernel"]) is not None and c["N"] == 128:
            e["traffic"] = TRAFFIC_PER_ROW[e["kernel"]] * n
    roof = max(kernels, key=lambda e: e["step_ms"])
    forms = {prec: {"frames_per_s": value, "fit_s": fit_s, "recon_frames_per_s": K / rec_s}}
    if not args.no_forms:
        other = "fp32" if prec == "mixed" else "mixed"
        forms[other] = time_form(sc, c, dmd, dev, st, other, out, ks)
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3" if prec == "mixed" else "f32",
        "data": "synthetic", "impl": "ours",
        "config": {"workload": c["workload"], "n": n, "m": m, "r": r, "frames": K, "precision": prec,
                   "parallelism": f"replicas{world}", "l2": "inputs (5.06 GB) and outputs (25.2 GB) exceed L2"},
        "fit_s": fit_s, "recon_frames_per_s": K / rec_s, "recon_s": rec_s,
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
        "forms": forms, "kernels": kernels, "adjoint": adjoint, "optdmd": optdmd, "device": device_info(dev),
        "parity": {"status": model.status()},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config, sample_rows=args.cpu_rows)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batch_scenes(c, dev):
    """The many-scene workload: seeded sizes, snapshot counts and ranks."""
    from paper_2502_05339_gb300 import synth
    g = np.random.default_rng(c["seed"])
    items = []
    for i in range(c["scenes"]):
        N = int(round(np.exp(g.uniform(np.log(64), np.log(512)))))
        m = int(g.integers(50, 401))
        r = int(g.integers(5, 65)) * 2
        r = min(r, m - 2 - (m % 2))
        # frequencies stratified over (0, pi), the reading taken for the
        # rank-150 workload: with up to 64 pairs, U(0, pi/4) is not resolvable
        sc = synth.linear_modes_scene(N, 2, r // 2, m, c["seed"] * 1000 + i, sigma_lo=-0.05, omega_hi=math.pi,
                                      stratified=True, noise=1e-5, device=dev)
        items.append([sc.S, sc.n, r, c["seed"] + i, list(range(c["frames"]))])
    return items


def resolvable_ranks(items, dmd):
    """A drawn scene could carry modes below what the fit resolves (the fit
    then reports DMD_ERANK).  Before timing, each scene is fitted in both
    forms and its rank lowered in steps of 2 until both fit it; with the
    shifted CholeskyQR fallback no scene of the workload needs it, and the
    number lowered is reported."""
    for it in items:
        S, n, r, seed, _ = it
        while r > 2:
            ok = True
            for prec in ("fp32", "mixed"):
                mdl = dmd.dmd_fit(S, n, r, oversample=10, power_iters=2, precision=prec, seed=seed)
                torch.cuda.synchronize()
                ok = ok and mdl.status() == 0
            if ok:
                break
            r -= 2
        it[2] = r
    return [tuple(it) for it in items]


def run_batch(args):
    """Batched fit + predict of many scenes (one dmd_fit_predict_batch call per step)."""
    from paper_2502_05339_gb300 import dmd
    dev = torch.device("cuda", torch.cuda.current_device())
    c = CONFIGS[args.config]
    drawn = batch_scenes(c, dev)
    drawn_ranks = [it[2] for it in drawn]
    items = resolvable_ranks(drawn, dmd)
    lowered = sum(1 for a, it in zip(drawn_ranks, items) if it[2] != a)
    batch = dmd.Batch(items, lanes=16, precision=args.precision)
    st = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    for mdl in batch.models:
        mdl.check()
    # the batch captured once as a CUDA graph (the library's launches recorded
    # into it), then one graph launch per step: no per-kernel host work
    launches0 = dmd.lib().dmd_launch_count()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        batch.run()
    in_graph = dmd.lib().dmd_launch_count() - launches0
    st = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.steps):
            graph.replay()
        b.record(st)
        torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    for mdl in batch.models:
        mdl.check()
    # the same batch called directly (every kernel launched from the host)
    direct = event_time(lambda: batch.run(), st, reps=args.steps)
    serial = event_time(lambda: [batch_one(dmd, it, args.precision) for it in items], st, reps=1)
    line = {"metric": "batched DMD fit + 256-frame prediction, scenes/s (many-scene workload)",
            "value": c["scenes"] * args.steps / sec, "unit": "scenes/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3" if args.precision == "mixed" else "f32",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": c["workload"], "precision": args.precision, "lanes": 16,
                       "rows_total": int(sum(it[1] for it in items)), "ranks": [int(it[2]) for it in items],
                       "ranks_lowered": lowered},
            "launch": "one CUDA graph per step (the batch captured once)",
            "direct_call_s": direct, "direct_call_scenes_per_s": c["scenes"] / direct,
            "one_scene_at_a_time_s": serial, "gpu_launches": int(in_graph),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_dmdc(args):
    """DMD with control: fit, 200-step controlled rollout to one frame, and
    the adjoint of ||x_200 - x_target||^2 w.r.t. the inputs and b."""
    from paper_2502_05339_gb300 import dmd, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    c = CONFIGS[args.config]
    prec = args.precision
    sc = synth.config2(seed=c["seed"], device=dev)
    st = torch.cuda.current_stream(dev)
    Ups = torch.as_tensor(sc.extra["U"].T.astype(np.float32)).contiguous().to(dev)      # (m, q)
    g = np.random.default_rng(c["seed"])
    T = c["rollout"]
    u = torch.as_tensor(synth.piecewise_controls(g, c["q"], T).T.astype(np.float32)).contiguous().to(dev)
    # The recipe's weakest latent direction sits at sigma_100 / sigma_1 ~ 6e-6,
    # below what the first CholeskyQR pass resolves: the fit takes the shifted
    # fallback and fits the stated rank.
    r = c["r"]
    fit = lambda: dmd.dmd_fit(sc.S, sc.n, r, oversample=c["oversample"], power_iters=c["power_iters"],
                              precision=prec, seed=c["seed"], Ups=Ups)
    model = fit()
    torch.cuda.synchronize()
    model.check()
    for _ in range(args.warmup - 1):
        fit()
    fit_s = event_time(fit, st, reps=max(1, args.steps))
    tgt = torch.zeros(model.ldPhi, dtype=torch.float32, device=dev)
    w = torch.ones(1, dtype=torch.float64, device=dev)
    fwd = event_time(lambda: dmd.dmd_predict(model, [T], u=u, precision=prec), st)
    loss = event_time(lambda: dmd.dmd_predict_loss(model, [T], tgt, w, u=u, precision=prec), st)
    grad = event_time(lambda: dmd.dmd_predict_loss(model, [T], tgt, w, want_grad=True, u=u, precision=prec), st)
    line = {"metric": "DMDc fit seconds (96^3 x 3, m=300, q=8, r=100)", "value": fit_s, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * fit_s,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec == "mixed" else "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": c["workload"], "n": sc.n, "precision": prec, "r": r},
            "rollout_frame_s": fwd, "loss_s": loss, "loss_and_grad_s": grad, "grad_over_forward": grad / loss,
            "parity": {"status": model.status()}}
    print(json.dumps(line), flush=True)


def run_upsample(args):
    """Upsampling evolution: T frames H_t = Phi_R C_t from H_0 and T inputs
    (one dmd_upsample call per step: the model's Gram, one tall reduction of
    the inputs, the FP64 projection and the closed-form evolution, one tall
    product)."""
    from paper_2502_05339_gb300 import dmd, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    c = CONFIGS[args.config]
    prec = args.precision
    sc = synth.config1(seed=c["seed"], device=dev)
    st = torch.cuda.current_stream(dev)
    model = dmd.dmd_fit(sc.S, sc.n, c["r"], oversample=c["oversample"], power_iters=c["power_iters"],
                        precision=prec, seed=c["seed"])
    torch.cuda.synchronize()
    model.check()
    T = c["frames"]
    coarse = synth.linear_modes_scene(c["coarse"], 3, 75, T, c["seed"] + 7, sigma_lo=-0.02, omega_hi=math.pi,
                                      stratified=True, device=dev)
    inp = synth.prolong(coarse.S, c["coarse"], 3, c["N"] // c["coarse"])
    del coarse
    assert inp.shape[1] == model.ldPhi
    inp[0] = sc.S[0, :model.ldPhi]
    del sc
    torch.cuda.empty_cache()
    out = torch.empty((T, model.ldPhi), dtype=torch.float32, device=dev)
    info = torch.zeros(8, dtype=torch.int32, device=dev)
    gram = torch.empty((model.r, model.r), dtype=torch.float64, device=dev)
    # the model's Gram Phi_R^T Phi_R depends on the model only: formed by the
    # first call, reused by the timed ones (the per-call cost with it is
    # reported beside the value)
    full = lambda: dmd.dmd_upsample(model, inp, c["threshold"], precision=prec, out=out, info=info, gram=gram)
    call = lambda: dmd.dmd_upsample(model, inp, c["threshold"], precision=prec, out=out, info=info, gram=gram,
                                    gram_given=True)
    with_gram_s = event_time(full, st, reps=2)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    if int(info[0].item()) != 0:
        raise RuntimeError(f"dmd_upsample: device status {info.cpu().tolist()}")
    launches0 = dmd.lib().dmd_launch_count()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.steps):
            call()
        b.record(st)
        torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3 / args.steps
    n, r = model.n, model.r
    algo = 4.0 * n * (T + 1) + 4.0 * n * T + 2 * 4.0 * n * r   # inputs, outputs, Phi_R (reduction, product)
    peaks, peak_kind = load_peaks()
    low = int(np.sum(np.abs(np.angle(model.lam())) < c["threshold"]))
    line = {"metric": "upsampled frames/s (Sec. 6.3.1, 128^3 x 3, r=150)", "value": T / sec, "unit": "frames/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec == "mixed" else "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": c["workload"], "n": n, "r": r, "frames": T, "low_order_modes": low,
                       "precision": prec, "l2": "inputs (25.2 GB) and outputs (25.2 GB) exceed L2"},
            "roofline": {"bound": "hbm", "achieved": algo / sec / 1e9, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": algo / sec / 1e9 / peaks["hbm_gbs"], "traffic": None,
                         "peak_source": peak_kind,
                         "algorithmic": "4n(T+1) input + 4nT output + 2 x 4nr Phi_R bytes per call"},
            "with_model_gram_s": with_gram_s, "with_model_gram_frames_per_s": T / with_gram_s,
            "gpu_launches": int((dmd.lib().dmd_launch_count() - launches0) // max(args.steps, 1)),
            "clocks": clk.summary(), "parity": {"status": int(info[0].item())}}
    print(json.dumps(line), flush=True)


def run_advect(args):
    """Density advection: K steps per call (velocity frames rebuilt in batches
    by the reconstruction product, one semi-Lagrangian launch per step)."""
    from paper_2502_05339_gb300 import dmd, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    c = CONFIGS[args.config]
    prec = args.precision
    sc = synth.config1(seed=c["seed"], device=dev)
    st = torch.cuda.current_stream(dev)
    model = dmd.dmd_fit(sc.S, sc.n, c["r"], oversample=c["oversample"], power_iters=c["power_iters"],
                        precision=prec, seed=c["seed"])
    torch.cuda.synchronize()
    model.check()
    del sc
    torch.cuda.empty_cache()
    N, K = c["N"], c["frames"]
    ax = (torch.arange(N, dtype=torch.float64, device=dev) + 0.5) / N
    x, y, z = torch.meshgrid(ax, ax, ax, indexing="ij")
    rho0 = (1.0 + 0.5 * torch.cos(2 * math.pi * x) * torch.sin(4 * math.pi * z)
            + 2.0 * torch.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / (2 * 0.125 ** 2)))
    rho0 = rho0.to(torch.float32).reshape(-1).contiguous()
    out = torch.empty((K + 1, dmd.round_up(N ** 3, 32)), dtype=torch.float32, device=dev)
    call = lambda: dmd.dmd_advect_density(model, rho0, N, 3, K, c["dt"], precision=prec, chunk=c["chunk"], out=out)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    launches0 = dmd.lib().dmd_launch_count()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.steps):
            call()
        b.record(st)
        torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3 / args.steps
    n, r, cells = model.n, model.r, N ** 3
    # velocity frames written and read once, density read and written per step, Phi_R per batch
    algo = K * (8.0 * n + 8.0 * cells) + math.ceil(K / c["chunk"]) * 4.0 * n * r
    peaks, peak_kind = load_peaks()
    line = {"metric": "density advection steps/s in the DMD velocity (Sec. 7.2, 128^3 x 3, r=150)",
            "value": K / sec, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec == "mixed" else "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": c["workload"], "n": n, "r": r, "steps_per_call": K, "precision": prec,
                       "l2": "velocity frames (25.2 MB each, 6.4 GB per batch) and densities exceed L2"},
            "roofline": {"bound": "hbm", "achieved": algo / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": algo / sec / 1e9 / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_kind,
                         "algorithmic": "per step 4n velocity written + 4n read + 8 N^3 density; 4nr Phi_R per batch"},
            "density_mass_drift": float((out[K, :cells].double().sum() / out[0, :cells].double().sum() - 1).item()),
            "gpu_launches": int((dmd.lib().dmd_launch_count() - launches0) // max(args.steps, 1)),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_large(args):
    """The large workload: a step is the fit of the 256^3 x 3 snapshots (60.6 GB)
    plus the streamed loss over 2000 frames and its gradient (frames never
    stored); value = frames / s of whole steps.  Mixed form only (the FP32
    form's CUDA-core products at this size are not a tensor-core measurement).
    The loss-gradient call is the dominant kernel: its roofline is in TFLOP/s
    of the BF16x3 products it executes (3 bf16 products per product of the
    method: forward 2 n r K and backward 2 n r K flops each) against the
    sustained dense bf16 peak, since it runs inside a long step."""
    from paper_2502_05339_gb300 import dmd, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    c = CONFIGS["cfg4"]
    prec = "mixed"
    t_gen = time.perf_counter()
    sc = synth.config4(seed=c["seed"], device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    n, m, K = sc.n, sc.m, c["frames"]
    st = torch.cuda.current_stream(dev)
    L = dmd.lib()
    # a drawn pair can sit below what the fit resolves: lower r in steps of 2 (at most 10)
    r = c["r"]
    while True:
        model = dmd.dmd_fit(sc.S, n, r, oversample=c["oversample"], power_iters=c["power_iters"], precision=prec,
                            seed=c["seed"])
        torch.cuda.synchronize()
        if model.status() == 0 or r <= c["r"] - 10:
            break
        r -= 2
    model.check()
    ks = torch.arange(K, dtype=torch.int32, device=dev)
    target = sc.S[0].clone()
    w = torch.as_tensor(np.random.default_rng(c["seed"]).uniform(0.0, 1.0, K)).to(dev)
    holder = {}

    def fit():
        holder["model"] = dmd.dmd_fit(sc.S, n, r, oversample=c["oversample"], power_iters=c["power_iters"],
                                      precision=prec, seed=c["seed"])

    def loss_grad():
        holder["res"] = dmd.dmd_predict_loss(holder["model"], ks, target, w, want_grad=True, precision=prec)

    def step():
        fit()
        loss_grad()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    holder["model"].check()
    fit_s = event_time(fit, st, reps=2)
    lg_s = event_time(loss_grad, st, reps=2)
    loss_s = event_time(lambda: dmd.dmd_predict_loss(holder["model"], ks, target, w, precision=prec), st, reps=2)
    launches0 = L.dmd_launch_count()
    torch.cuda.synchronize()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(st)
        for _ in range(args.steps):
            step()
        t1.record(st)
        torch.cuda.synchronize()
    elapsed = t0.elapsed_time(t1) / 1e3
    launches = (L.dmd_launch_count() - launches0) // max(args.steps, 1)
    peaks, peak_kind = load_peaks()
    sustained = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
    fl_grad = 3 * 4.0 * n * r * K
    fl_loss = 3 * 2.0 * n * r * K
    roof = {"kernel": "k_umma_loss_grad (streamed loss + gradient, 2000 frames)", "bound": "tensor",
            "achieved": fl_grad / lg_s / 1e12, "peak": sustained, "unit": "TFLOP/s",
            "frac": fl_grad / lg_s / 1e12 / sustained, "traffic": None,
            "peak_source": f"{peak_kind} bf16 dense, sustained", "launch_ms": 1e3 * lg_s,
            "algorithmic": "3 bf16 products x (2 n r K forward + 2 n r K backward) flops; timed around the "
                           "dmd_predict_loss call (the kernel plus the coefficient, partial-sum and chain-rule "
                           "launches)"}
    loss_entry = {"kernel": "k_umma_nn_ares<loss> (streamed loss alone)", "bound": "tensor",
                  "achieved": fl_loss / loss_s / 1e12, "peak": sustained, "unit": "TFLOP/s",
                  "frac": fl_loss / loss_s / 1e12 / sustained, "launch_ms": 1e3 * loss_s,
                  "algorithmic": "3 bf16 products x 2 n r K flops"}
    line = {
        "metric": "streamed loss+gradient frames/s, 256^3 x 3, r=150, 2000 frames (fit + loss + grad per step)",
        "value": K * args.steps / elapsed, "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic", "impl": "ours",
        "config": {"workload": c["workload"], "n": n, "m": m, "r": r, "frames": K, "precision": prec,
                   "l2": "snapshots (60.6 GB) and modes (30.2 GB) exceed L2"},
        "fit_s": fit_s, "loss_s": loss_s, "loss_and_grad_s": lg_s, "grad_over_loss": lg_s / loss_s,
        "e2e": None, "e2e_note": "not measured for this configuration: one step would copy 60.6 GB of snapshots",
        "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": roof, "kernels": [roof, loss_entry],
        "scene_generation_s": t_gen, "loss": float(holder["res"][0].item()),
        "parity": {"status": holder["model"].status(), "tests": "tests/test_gpu_config4.py"},
        "device": device_info(dev),
    }
    print(json.dumps(line), flush=True)


def batch_one(dmd, item, prec):
    S, n, r, seed, ks = item
    model = dmd.dmd_fit(S, n, r, oversample=10, power_iters=2, precision=prec, seed=seed)
    return dmd.dmd_predict(model, ks, precision=prec)


def adjoint_timing(model, ks, out, dmd, st, prec, rec_s):
    """Adjoint of the prediction against the forward: dmd_predict_backward of
    the stored frames (dL/dF taken as the frame buffer itself), and the
    streamed loss L = sum_k 0.5 ||x_k - x_0||^2 with and without its gradient
    (frames never stored: recomputed on the tensor cores in the mixed form, in
    stored chunks of 50 in the FP32 form)."""
    K = int(ks.numel())
    bwd = event_time(lambda: dmd.dmd_predict_backward(model, ks, out, precision=prec), st)
    target = out[0].clone()
    w = torch.ones(K, dtype=torch.float64, device=out.device)
    loss = event_time(lambda: dmd.dmd_predict_loss(model, ks, target, w, want_grad=False, precision=prec), st)
    grad = event_time(lambda: dmd.dmd_predict_loss(model, ks, target, w, want_grad=True, precision=prec), st)
    return {"forward_s": rec_s, "backward_s": bwd, "backward_over_forward": bwd / rec_s,
            "streamed_loss_s": loss, "streamed_loss_and_grad_s": grad, "grad_over_loss": grad / loss}


def optdmd_timing(S, n, c, dmd, st, prec, exact_fit_s):
    """OptDMD fit (Sec. 4.2) of the same snapshots: the exact fit's randomized
    SVD, then the device-side variable-projection loop and one tall lift."""
    stats = torch.zeros(4, dtype=torch.float64, device=S.device)
    holder = {}

    def fit():
        holder["m"] = dmd.dmd_fit_optdmd(S, n, c["r"], oversample=c["oversample"], power_iters=c["power_iters"],
                                         precision=prec, seed=c["seed"], stats=stats)

    sec = event_time(fit, st, reps=2)
    holder["m"].check()
    f0, f, evals, acc = stats.cpu().tolist()
    return {"fit_s": sec, "over_exact_fit": sec / exact_fit_s, "evaluations": int(evals), "accepted": int(acc),
            "objective_start": f0, "objective_end": f}


def device_info(dev):
    props = torch.cuda.get_device_properties(dev)
    free, total = torch.cuda.mem_get_info(dev)
    return {"name": props.name, "sms": props.multi_processor_count, "hbm_bytes": int(total),
            "hbm_free_bytes_at_end": int(free)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def gpu_local_cpus(dev):
    """Host CPUs of the GPU's own NUMA node (sysfs local_cpulist of its PCI
    function), or None when the system does not say."""
    try:
        p = torch.cuda.get_device_properties(dev)
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bdf}/local_cpulist") as f:
            text = f.read().strip()
        cpus = set()
        for part in text.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except (OSError, ValueError, AttributeError, RuntimeError):
        return None


def run_e2e(args, sc, c, dmd, dev, st, out, ks):
    """Same step through the public API with HOST snapshots in and HOST frames out.
    The pinned host buffers are allocated and first touched from the CPUs of
    the GPU's own NUMA node when the system names them (what a host
    application placing its buffers next to the GPU does)."""
    n, K = sc.n, c["frames"]
    old_aff = os.sched_getaffinity(0)
    local = gpu_local_cpus(dev)
    if local:
        os.sched_setaffinity(0, local)
    try:
        return _run_e2e(args, sc, c, dmd, dev, st, out, ks, local)
    finally:
        os.sched_setaffinity(0, old_aff)


def _run_e2e(args, sc, c, dmd, dev, st, out, ks, local):
    """Whole steps through the public API with the snapshots uploaded from and
    the frames downloaded to pinned host memory, pipelined over three streams:
    while the frames of step s come down (download stream), the snapshots of
    step s + 1 go up (upload stream) and step s + 1 is fitted and
    reconstructed (compute stream), with two device buffers of each kind.
    Every step's own upload and download are in the timed region; only the
    first upload and the last download are not overlapped.  (Measured on this
    node: ~193 GB/s device-to-host, ~211 GB/s host-to-device, ~341 GB/s both
    at once; one copy per direction reaches them.)"""
    n, K = sc.n, c["frames"]
    try:
        S_host = torch.empty(sc.S.shape, dtype=torch.float32, pin_memory=True)
        S_host.copy_(sc.S.cpu())
        F_host = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
    except RuntimeError as e:
        return {"value": None, "unit": "frames/s", "error": f"pinned host buffers: {e}"}
    S_dev = [torch.empty_like(sc.S), torch.empty_like(sc.S)]
    outs = [out, torch.empty_like(out)]
    steps = max(2, args.steps)
    up, comp, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    kt = ks if isinstance(ks, torch.Tensor) else torch.as_tensor(ks, dtype=torch.int32, device=dev)
    ev = lambda: torch.cuda.Event()
    fit_done = [None, None]     # S_dev[b] consumed by the fit of the step that used it
    down_done = [None, None]    # outs[b] downloaded

    def step(i):
        b = i % 2
        if fit_done[b] is not None:
            up.wait_event(fit_done[b])
        with torch.cuda.stream(up):
            S_dev[b].copy_(S_host, non_blocking=True)
        uploaded = ev()
        uploaded.record(up)
        comp.wait_event(uploaded)
        if down_done[b] is not None:
            comp.wait_event(down_done[b])
        with torch.cuda.stream(comp):
            model = dmd.dmd_fit(S_dev[b], n, c["r"], oversample=c["oversample"], power_iters=c["power_iters"],
                                precision=args.precision, seed=c["seed"])
            fit_done[b] = ev()
            fit_done[b].record(comp)
            dmd.dmd_predict(model, kt, precision=args.precision, out=outs[b])
        ready = ev()
        ready.record(comp)
        down.wait_event(ready)
        with torch.cuda.stream(down):
            F_host.copy_(outs[b], non_blocking=True)
        down_done[b] = ev()
        down_done[b].record(down)

    step(0)                                  # warm-up: allocator, library set-up
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    z = torch.cuda.Event(enable_timing=True)
    a.record(up)
    comp.wait_event(a)
    down.wait_event(a)
    for i in range(steps):
        step(i)
    z.record(down)
    torch.cuda.synchronize()
    sec = a.elapsed_time(z) / 1e3
    return {"value": K * steps / sec, "unit": "frames/s", "h2d_bytes_per_step": int(S_host.numel() * 4),
            "d2h_bytes_per_step": int(F_host.numel() * 4), "steps": steps,
            "host_cpus": f"{len(local)} GPU-local" if local else "unrestricted",
            "copies": "steps pipelined: upload and fit of step s+1 under the download of step s",
            "bytes_over_step_gbs": (S_host.numel() + F_host.numel()) * 4 * steps / sec / 1e9}


# DRAM bytes per row of n (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch divided by its rows) from the ncu captures of the 1,048,576-row cases
# summarised in profiles/tall_kernels_cfg1_1M_rows.md; traffic grows in
# proportion to the rows, so a full launch moves these x n bytes.
GRAM_TRAFFIC_PER_ROW = (1.002e9 + 0.154e9) / 1048576   # k_gram_f32: S once + the FP64 partials' read-modify-writes
TRAFFIC_PER_ROW = {
    "k_gram_f32 (snapshot Gram W = S^T S)": GRAM_TRAFFIC_PER_ROW,
    "k_umma_tn (projection Q1^T S)": 1.596e9 / 1048576,
    "k_umma_tn (Gram Q1^T Q1)": 0.737e9 / 1048576,
    "k_umma_nn_bres (sketch Q1 = X M)": None,   # kernel changed since its capture (converters, ring depth)
    "k_umma_nn_ares (reconstruction Phi_R C)": 4.786e9 / 1048576,
}


def alu_peak(peaks):
    """FP32 FFMA peak: 152 SMs x 128 lanes x 2 flops x maximum SM clock."""
    return 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def hbm_entry(name, bytes_, sec, launches, peaks, peak_kind, what):
    achieved = bytes_ / sec / 1e9
    peak = float(peaks["hbm_gbs"])
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": peak_kind, "launch_ms": 1e3 * sec,
            "launches_per_step": launches, "step_ms": 1e3 * sec * launches, "algorithmic": what}


def alu_entry(name, flops, sec, launches, peaks, what):
    achieved = flops / sec / 1e12
    peak = alu_peak(peaks)
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock", "launch_ms": 1e3 * sec,
            "launches_per_step": launches, "step_ms": 1e3 * sec * launches, "algorithmic": what}


def roofline(n, r, K, rec_s, prec, peaks, peak_kind):
    """Reconstruction launch F = Phi_R C (timed with events around dmd_predict)."""
    if prec == "mixed":
        return hbm_entry("k_umma_nn_ares (reconstruction Phi_R C)", 4.0 * n * (r + K), rec_s, 1, peaks, peak_kind,
                         "4 n (r + K) bytes: Phi_R read once, K frames written")
    return alu_entry("k_gemm_nn_f32 (reconstruction Phi_R C)", 2.0 * n * r * K, rec_s, 1, peaks,
                     "2 n r K flops")


def event_time(fn, st, reps=3):
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def kernel_rooflines(sc, c, dmd, dev, st, prec, peaks, peak_kind):
    """The fit's tall passes, each launched alone on the step's own shapes
    (same kernels, same sizes) and timed with CUDA events on the launching
    stream: the snapshot Gram W = S^T S, the sketch product Q1 = X M, the
    tensor-core reductions Q1^T Q1 and Q1^T S (mixed form; the FP32 form runs
    them on the CUDA cores).  One fit forms one tall sketch (the power
    iterations run in the snapshot-Gram space), then its Gram and the
    projection; the sketch kernel runs again for the modes X' M_R."""
    n, m, r = sc.n, sc.m, c["r"]
    l = min(r + c["oversample"], m)
    S, ld = sc.S, sc.S.shape[1]
    X = S[:m]
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    Q = torch.randn((l, ld), device=dev, generator=g)
    M = torch.randn((l, m), dtype=torch.float64, device=dev, generator=g)
    out = []
    sec = event_time(lambda: dmd.dmd_gemm_tn(S, S, n, precision="fp32"), st)
    out.append(alu_entry("k_gram_f32 (snapshot Gram W = S^T S)", float(n) * (m + 1) * (m + 2), sec, 1, peaks,
                         "n (m+1)(m+2) flops: 2n per distinct entry of the symmetric W"))
    npass = 1
    sec = event_time(lambda: dmd.dmd_gemm_tall(X, n, M, precision=prec, out=Q), st)
    name = "k_umma_nn_bres (sketch Q1 = X M)" if prec == "mixed" else "k_gemm_nn_f32 (sketch Q1 = X M)"
    if prec == "mixed":
        out.append(hbm_entry(name, 4.0 * n * (m + l), sec, npass + 1, peaks, peak_kind,
                             "4 n (m + l) bytes: X read, Q1 written (also the modes X' M_R)"))
    else:
        out.append(alu_entry(name, 2.0 * n * m * l, sec, npass + 1, peaks, "2 n m l flops"))
    sec = event_time(lambda: dmd.dmd_gemm_tn(Q, Q, n, precision=prec), st)
    name = "k_umma_tn (Gram Q1^T Q1)" if prec == "mixed" else "k_gemm_tn_f32 (Gram Q1^T Q1)"
    if prec == "mixed":
        out.append(hbm_entry(name, 4.0 * n * l, sec, npass, peaks, peak_kind, "4 n l bytes: Q1 read once"))
    else:
        out.append(alu_entry(name, float(n) * l * (l + 1), sec, npass, peaks, "n l (l+1) flops"))
    sec = event_time(lambda: dmd.dmd_gemm_tn(Q, S, n, precision=prec), st)
    name = "k_umma_tn (projection Q1^T S)" if prec == "mixed" else "k_gemm_tn_f32 (projection Q1^T S)"
    if prec == "mixed":
        out.append(hbm_entry(name, 4.0 * n * (l + m + 1), sec, npass, peaks, peak_kind,
                             "4 n (l + m + 1) bytes: Q1 and S read once"))
    else:
        out.append(alu_entry(name, 2.0 * n * l * (m + 1), sec, npass, peaks, "2 n l (m+1) flops"))
    del Q, M
    torch.cuda.empty_cache()
    return out


def time_form(sc, c, dmd, dev, st, prec, out, ks):
    """Fit seconds, reconstruction frames/s and whole-step frames/s of one form."""
    n, K = sc.n, c["frames"]
    fit = lambda: dmd.dmd_fit(sc.S, n, c["r"], oversample=c["oversample"], power_iters=c["power_iters"],
                              precision=prec, seed=c["seed"])
    model = fit()
    torch.cuda.synchronize()
    model.check()
    fit_s = event_time(fit, st)
    rec_s = event_time(lambda: dmd.dmd_predict(model, ks, precision=prec, out=out), st)
    return {"frames_per_s": K / (fit_s + rec_s), "fit_s": fit_s, "recon_frames_per_s": K / rec_s}


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
            "cpu": cpu_model(),
            "sample": f"{sc.name}: n={sc.n} rows ({sc.n / n_full:.4f} of the workload), m={c['m']}, r={c['r']}, "
                      f"{c['frames']} frames; EXTRAPOLATED: the times measured on this sample are scaled "
                      f"linearly by n (x{scale:.0f}; fit O(n m^2), prediction O(n r K)) to fit {fit_s:.1f} s and "
                      f"predict {pred_s:.1f} s at full n",
            "extrapolated": scale != 1.0, "scale_by_n": scale, "measured_s": t2 - t0}


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


# ---------------------------------------------------------------------------
# small cases of single kernels, for profilers (--case NAME [--rows N])
#
# Each case builds seeded random operands of the 128^3 x 3 workload's column
# counts on cuda:0 with a reduced row count (default 1,048,576 rows: every
# operand still exceeds the 129 MB L2, the whole case holds a few GB) and calls
# the same entry point twice, so a profiler can skip the first (warm-up) launch:
#
#   gram    snapshot Gram W = S^T S on the CUDA cores (201 columns, symmetric)
#   tn      tensor-core reduction Q^T S (160 x 201 columns, BF16x3)
#   gramq   tensor-core Gram Q^T Q (160 columns, BF16x3)
#   sketch  tensor-core tall product X M (200 -> 160 columns, BF16x3)
#   recon   reconstruction Phi_R C of 1000 frames (150 modes, BF16x3)
#   loss    streamed quadratic loss of 250 frames (150 modes, BF16x3; frames
#           never stored: the reconstruction kernel's loss epilogue)
#   lossgrad  the same loss with its gradient (the fused loss-gradient kernel)
#   advect  density advection (Sec. 7.2) on a 128^3 grid: a random 150-mode
#           velocity model (RMS ~0.5 cells per unit step), 64 steps, frames
#           rebuilt in batches of 64 (rows fixed by the grid; --rows is ignored)
#   optdmd  OptDMD fit (Sec. 4.2) of a 3D 70^3 x 3 linear-modes scene (1,029,000
#           rows; 200 snapshots, 75 pairs with stratified frequencies, rank 150,
#           BF16x3 tall passes): the small FP64 loop is independent of the rows
# ---------------------------------------------------------------------------

CASE_M, CASE_L, CASE_R, CASE_FRAMES = 200, 160, 150, 1000


def _case_rand(rows, cols, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randn((cols, rows), device="cuda", generator=g)


def _case_model(rows):
    P = _case_rand(rows, CASE_R, 3)
    rng = np.random.default_rng(4)
    lam = np.exp(rng.uniform(-0.02, 0, CASE_R // 2) + 1j * rng.uniform(0, np.pi, CASE_R // 2))
    modal = np.zeros(4 * CASE_R)
    modal[0:CASE_R:2], modal[1:CASE_R:2] = lam.real, lam.real
    modal[CASE_R:2 * CASE_R:2], modal[CASE_R + 1:2 * CASE_R:2] = lam.imag, -lam.imag
    modal[2 * CASE_R:3 * CASE_R] = rng.standard_normal(CASE_R)
    from paper_2502_05339_gb300 import dmd
    return dmd.DmdModel(P, torch.as_tensor(modal).cuda(), torch.zeros(8, dtype=torch.int32, device="cuda"),
                        rows, CASE_R, 0)


def run_case(case: str, rows: int, reps: int = 2):
    from paper_2502_05339_gb300 import dmd
    dmd.lib()
    if case == "gram":
        S = _case_rand(rows, CASE_M + 1, 1)
        for _ in range(reps):
            dmd.dmd_gemm_tn(S, S, rows, precision="fp32")
    elif case in ("tn", "gramq"):
        Q = _case_rand(rows, CASE_L, 2)
        S = Q if case == "gramq" else _case_rand(rows, CASE_M + 1, 1)
        for _ in range(reps):
            dmd.dmd_gemm_tn(Q, S, rows, precision="mixed")
    elif case == "sketch":
        X = _case_rand(rows, CASE_M, 1)
        M = torch.randn((CASE_L, CASE_M), dtype=torch.float64, device="cuda")
        for _ in range(reps):
            dmd.dmd_gemm_tall(X, rows, M, precision="mixed")
    elif case == "recon":
        model = _case_model(rows)
        ks = torch.arange(CASE_FRAMES, dtype=torch.int32, device="cuda")
        out = torch.empty((CASE_FRAMES, model.ldPhi), dtype=torch.float32, device="cuda")
        for _ in range(reps):
            dmd.dmd_predict(model, ks, precision="mixed", out=out)
    elif case in ("loss", "lossgrad"):
        model = _case_model(rows)
        ks = torch.arange(CASE_FRAMES // 4, dtype=torch.int32, device="cuda")
        target = torch.randn(model.ldPhi, device="cuda")
        w = torch.rand(ks.numel(), dtype=torch.float64, device="cuda")
        for _ in range(reps):
            dmd.dmd_predict_loss(model, ks, target, w, want_grad=case == "lossgrad", precision="mixed")
    elif case == "advect":
        N = 128
        model = _case_model(3 * N ** 3)
        model.Phi_R.mul_(0.05)
        rho0 = torch.rand(N ** 3, device="cuda")
        for _ in range(reps):
            dmd.dmd_advect_density(model, rho0, N, 3, 64, 0.5, precision="mixed", chunk=64)
    elif case == "optdmd":
        import math
        from paper_2502_05339_gb300 import synth
        sc = synth.linear_modes_scene(70, 3, CASE_R // 2, CASE_M, 1001, sigma_lo=-0.02, omega_hi=math.pi,
                                      stratified=True, noise=1e-4, nonlinear=1e-3, device="cuda")
        for _ in range(reps):
            dmd.dmd_fit_optdmd(sc.S, sc.n, CASE_R, precision="mixed", seed=1001).check()
    else:
        raise SystemExit(f"unknown case {case!r}")
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("DMD_BENCH_PRECISION", "mixed"), choices=["fp32", "mixed"])
    ap.add_argument("--no-forms", action="store_true", help="skip the side-by-side timing of the other form")
    ap.add_argument("--no-optdmd", action="store_true", help="skip the OptDMD fit timing")
    ap.add_argument("--no-kernels", action="store_true", help="skip the per-kernel roofline timings")
    ap.add_argument("--config", default="cfg1", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=None)
    ap.add_argument("--case", default=None, help="run one kernel's small profiling case and exit")
    ap.add_argument("--rows", type=int, default=1 << 20, help="rows of the --case operands")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.case:
        run_case(args.case, args.rows)
        print("ok", args.case, args.rows)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "cfg3":
        run_batch(args)
    elif args.config == "cfg2":
        run_dmdc(args)
    elif args.config == "up":
        run_upsample(args)
    elif args.config == "adv":
        run_advect(args)
    elif args.config == "cfg4":
        run_large(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
