"""Benchmark of the whole hot path: MNF fusion of every position's exposure bracket followed by
the iterative reconstruction, on the lab-scale workload (1024^2 object, 256^2 probe, 1600
Fermat-spiral positions, 5 exposures, 6 pyramid levels, 200 iterations), synthetic data.

One step = fuse_stack over all positions + ptycho_init + ptycho_iterate(200) + ptycho_destroy.
The metric is position-updates per second (one update = one position through patch extraction,
FFT, modulus replacement, inverse FFT and the object/probe updates, in one iteration); fusion
and set-up time count against it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (it is the only reference that exists: the paper publishes no code or timings).
Under torchrun each rank reconstructs its own independent scan (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "position-updates/s"
WORKLOAD = "lab"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["lab", "mixed", "wide64", "wide128", "batched", "warm"], default="lab",
                    help="lab: coherent lab-scale scan (the headline); mixed: the same scan with "
                         "8 incoherent probe modes, 100 iterations; wide64: 64^2 probe, 9216 "
                         "raster positions on a 1024^2 object, 50 iterations; wide128: 128^2 probe, "
                         "2304 positions, 50 iterations; batched: 64 uneven "
                         "datasets (N in {64, 128, 256}, 49-900 positions) in one batch, 50 iterations; warm: "
                         "train the warm-start network, then time to NRMSE from it vs the flat object")
    ap.add_argument("--fft", choices=["radix_fp32", "dftgemm_bf16x3"], default="radix_fp32",
                    help="FFT form of the exit-wave step (dftgemm_bf16x3: tensor cores, N = 64, 128, 256)")
    ap.add_argument("--iters", type=int, default=None,
                    help="override the iteration count (profiling runs only; not a bench value)")
    ap.add_argument("--positions", type=int, default=None,
                    help="use only the first N scan positions (profiling runs only; not a bench value)")
    ap.add_argument("--warm-objects", type=int, default=None,
                    help="warm workload: training objects per scale (profiling runs only)")
    ap.add_argument("--warm-epochs", type=int, default=None,
                    help="warm workload: epochs per scale (profiling runs only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-nrmse", action="store_true")
    ap.add_argument("--nrmse-iters", type=int, default=400)
    return ap.parse_args()


def rank_seed(base: int, rank: int) -> int:
    """Each rank reconstructs its own independent scan (weak scaling)."""
    return base + 7919 * rank


def max_over_ranks(value: float, dist, device) -> float:
    """The job's time is the slowest rank's; no data-path collective is involved."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
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
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = [s for s in sm if s >= 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(hi), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def fuse_launches(levels: int) -> int:
    # reduce0 + (L-2) reduces + base + (L-1) collapses; L = 1: base only
    return 1 if levels == 1 else 2 * levels - 1


def exit_wave_bytes_per_position(N: int) -> int:
    """Algorithmic bytes of one position through the exit-wave kernel: amplitudes A_j (4 N^2),
    object patch (8 N^2) and probe (8 N^2) read, psi_j' (8 N^2) written."""
    return 28 * N * N


def exit_wave_flops_per_position(N: int) -> float:
    """Two unitary 2-D FFTs (5 n log2 n each, n = N^2) plus ~20 flops per pixel for the
    probe-object product, the unitary scalings and the modulus replacement with its error."""
    n = N * N
    return 2 * 5.0 * n * np.log2(n) + 20.0 * n


def dftgemm_flops_per_position(N: int) -> float:
    """Tensor-core flops of the split-BF16 exit wave: 4 real GEMM passes, 3 split terms each.
    N = 64: the 128 x 128 real DFT matrix times the 128 x 64 interleaved operand of a patch.
    N = 128: the same 64-point matrix times two halves (even / odd samples) of 128 vectors.
    N = 256: the same matrix times the four decimated quarters (x[4 r + q]) of 256 vectors."""
    if N == 256:
        return 4 * 3 * 2.0 * 128 * 128 * (4 * 256)
    if N == 128:
        return 4 * 3 * 2.0 * 128 * 128 * 256
    return 4 * 3 * 2.0 * (2 * N) * (2 * N) * N


def bf16_peak_tflops():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    return 1800.0, "fallback"


def fp32_peak_tflops(sm_mhz: float) -> float:
    """Derived FP32 rate for context: 148 SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


def iteration_bytes_per_update(N: int) -> int:
    """Algorithmic bytes of one position-update through the whole iteration: A_j (4 N^2), the
    object patch (8 N^2), the object numerator read-modify-write (16 N^2) and the probe
    numerator (8 N^2) = 36 N^2."""
    return 36 * N * N


def iteration_flops_per_update(N: int) -> float:
    """Flops of one position-update through the whole iteration: two 2-D FFTs (5 n log2 n
    each, n = N^2) plus ~60 flops per pixel of pointwise work (exit wave, modulus, object and
    probe numerators and denominators, updates)."""
    n = N * N
    return 2 * 5.0 * n * np.log2(n) + 60.0 * n


# DRAM bytes per position of the N = 256 exit-wave kernel from one ncu capture (400 lab
# positions, one launch: dram__bytes_read.sum + dram__bytes_write.sum), valid only for the
# kernel sources it was taken on (their SHA-256, first 16 hex digits).  A changed kernel
# reports traffic null until it is captured again.
EXIT_TRAFFIC = {"sources_sha16": "7e0377b69d8cbf7c", "bytes_per_position": 2148216,
                "capture": "ncu, k_exit_wave_tma<16, FULL>, one launch over 888 lab positions = three whole rounds of 296 CTAs"}


def exit_kernel_sources_sha16() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("exit_tma.cuh", "fft.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_2608_01746_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------- batched arm
def run_batched(args, world, rank, local):
    """64 uneven datasets advanced together (ptycho_batch_*: multi-dataset exit-wave launches,
    concurrent per-dataset branches, CUDA graph, autotuned launch shapes).  One step = fusion of
    every dataset + ptycho_init of every dataset + batch creation + 50 iterations + teardown."""
    import torch
    from paper_2608_01746_b300 import api, synth

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    base = rank_seed(synth.seed_for("batched"), rank)
    cfgs = synth.batched_configs(seed=base)
    n_iter = args.iters or cfgs[0].n_iter
    scans = [synth.make_scan_torch(c, seed=base * 1000 + d, device=dev) for d, c in enumerate(cfgs)]
    params = [api.fuse_params(levels=c.levels, clip=float(c.clip)) for c in cfgs]
    fused = [torch.empty((c.n_pos, c.N, c.N), dtype=torch.float32, device=dev) for c in cfgs]
    obj0 = [torch.ones((c.M, c.M), dtype=torch.complex64, device=dev) for c in cfgs]
    probe0 = [torch.from_numpy(sc["probe"].astype(np.complex64)).to(dev) for sc in scans]
    stream = torch.cuda.current_stream(dev)
    J_all = [c.n_pos for c in cfgs]
    updates_per_iter = sum(J_all)

    def fft_for(c, fft):
        return fft

    def make_handles(fft, raws=None):
        for d, c in enumerate(cfgs):
            api.fuse_stack(scans[d]["raw"] if raws is None else raws[d], c.times, params[d], out=fused[d],
                           stream=stream)
        return [api.ptycho_init(fused[d], scans[d]["pos"], obj0[d], probe0[d], stream=stream,
                                fft_path=fft_for(c, fft)) for d, c in enumerate(cfgs)]

    def step(fft=args.fft, raws=None):
        hs = make_handles(fft, raws)
        b = api.ptycho_batch_create(hs, graph=True, autotune=True, stream=stream)
        api.ptycho_batch_iterate(b, n_iter, errors=False)
        api.ptycho_batch_destroy(b)
        return hs

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        for h in step():
            api.ptycho_destroy(h)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        for h in step():
            api.ptycho_destroy(h)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    updates = updates_per_iter * n_iter * args.steps * world
    value = updates / (ms_total / 1e3)

    # iterations only, per form: serial handles, plain batch, graph + autotune, other FFT form
    def iter_ms(mode, fft):
        hs = make_handles(fft)
        b = None
        if mode != "serial":
            b = api.ptycho_batch_create(hs, graph=mode in ("tuned", "one"), autotune=mode == "tuned",
                                        one_launch=mode == "one", stream=stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if b is None:
            for h in hs:
                api.ptycho_iterate(h, n_iter, errors=False)
            # each handle works on its own stream, ordered after `stream` only through init
            torch.cuda.synchronize(dev)
            e1.record(stream)
        else:
            api.ptycho_batch_iterate(b, n_iter, errors=False)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        desc = api.ptycho_batch_describe(b) if b is not None else None
        if b is not None:
            api.ptycho_batch_destroy(b)
        for h in hs:
            api.ptycho_destroy(h)
        return e0.elapsed_time(e1), desc

    variants = None
    if rank == 0:
        other = "dftgemm_bf16x3" if args.fft == "radix_fp32" else "radix_fp32"
        variants = {}
        for name, mode, fft in [("serial_handles", "serial", args.fft), ("batch_plain", "plain", args.fft),
                                ("batch_graph_autotuned", "tuned", args.fft),
                                ("batch_graph_one_launch", "one", args.fft),
                                (f"batch_graph_autotuned_{other}", "tuned", other)]:
            ms, desc = iter_ms(mode, fft)
            variants[name] = {"ms_per_iteration": round(ms / n_iter, 4),
                              "position_updates_per_s": round(updates_per_iter * n_iter / (ms / 1e3), 1)}
            if desc:
                variants[name]["autotune"] = json.loads(desc)

    e2e = None
    if not args.no_e2e:
        raws_h = [sc["raw"].cpu().pin_memory() for sc in scans]
        raws_d = [torch.empty_like(sc["raw"]) for sc in scans]
        outs = [np.empty((c.M, c.M), np.complex64) for c in cfgs]

        def e2e_step():
            for d in range(len(cfgs)):
                raws_d[d].copy_(raws_h[d], non_blocking=True)
            hs = step(raws=raws_d)
            for d, h in enumerate(hs):
                api.ptycho_get_object(h, outs[d])
                api.ptycho_destroy(h)

        e2e_step()
        barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - w0, dist, dev)
        e2e = {"value": round(updates / e2e_s, 1), "unit": METRIC,
               "h2d_bytes_per_step": int(sum(r.numel() * 2 for r in raws_h) + sum(sc["pos"].nbytes for sc in scans)
                                         + sum(o.nbytes for o in outs) + sum(p.numel() * 8 for p in probe0)),
               "d2h_bytes_per_step": int(sum(o.nbytes for o in outs))}

    # whole-iteration roofline (every kernel of the batched iteration together; per-kernel events
    # are not available inside the graph): 36 N^2 bytes per position-update against the measured
    # copy bandwidth, and the iteration's flops against the measured FP32 FMA rate
    it_ms = variants["batch_graph_autotuned"]["ms_per_iteration"] if variants else ms_total / args.steps / n_iter
    fma = api.measure_fp32_fma_tflops(device=dev)
    flops = sum(iteration_flops_per_update(c.N) * c.n_pos for c in cfgs) / (it_ms / 1e3) / 1e12
    hbm_peak, peak_kind = peaks()
    hbm = sum(iteration_bytes_per_update(c.N) * c.n_pos for c in cfgs) / (it_ms / 1e3) / 1e9
    roof = {"kernel": "whole batched iteration (all kernels; per-kernel events are not available inside the graph)",
            "bound": "hbm", "achieved": round(hbm, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(hbm / hbm_peak, 4), "peak_kind": peak_kind,
            "bytes_per_position_update": "36 N^2", "traffic": None, "avg_iteration_ms": round(it_ms, 4),
            "alu_view": {"achieved_tflops": round(flops, 2), "peak_tflops": round(fma["tflops"], 2),
                         "peak_kind": "measured: the library's FP32 FMA kernel, best of 5 launches",
                         "frac": round(flops / fma["tflops"], 4)}}
    by_n = {n: sum(1 for c in cfgs if c.N == n) for n in sorted({c.N for c in cfgs})}
    launches_per_iter = (len(by_n) - 1 + sum(1 for c in cfgs if c.N == 256)  # class launches + N=256 exits
                         + 2 * len(cfgs) + 3 * len(cfgs))   # object (2, the error inside), probe (3)
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.fft == "radix_fp32" else "bf16x3 (split) with f32 accumulate",
        "data": "synthetic (seeded jittered raster scans, Poisson counts, 12-bit clip)",
        "config": {"workload": (f"batched: 64 uneven datasets ("
                                + ", ".join(f"{v} with {n}^2 probes" for n, v in by_n.items()) + "), "
                                f"{updates_per_iter} positions in all, objects {min(c.M for c in cfgs)}-"
                                f"{max(c.M for c in cfgs)} px, 3 exposures, 4-level pyramid, {n_iter} iterations "
                                "per step, one batch (CUDA graph, autotuned)"),
                   "fft": args.fft, "datasets": len(cfgs), "positions": updates_per_iter,
                   "iterations": n_iter,
                   "l2": f"inputs larger than L2 (raw stacks {sum(sc['raw'].numel() for sc in scans) * 2 / 1e9:.2f} GB per step)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "variants_iterations_only": variants,
        "roofline": roof, "clocks": clk,
        "gpu_launches": int(args.steps * (len(cfgs) * (2 * cfgs[0].levels - 1 + 2) + n_iter * launches_per_iter)),
        "e2e": e2e, "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- warm start
def warm_flops_per_sample(layers, side):
    """Forward multiply-add flops of the warm-start network for one (side x side) input."""
    f = 0
    for cin, cout, mode in layers:
        side = side // 2 if mode == "s2" else (side * 2 if mode == "up" else side)
        f += 2 * 9 * cin * cout * side * side
    return f


def run_warm(args, world, rank, local):
    """The learned warm start at two scales: the network is trained on the GPU (tensor-core
    kernels) on scans of random objects, then the workload's own scan is reconstructed from the
    stitched prediction (kept only if the first-iteration judge prefers it) and from the flat
    object; time to the NRMSE goal (1e-2, else 1.05 x the better floor) counts inference,
    stitching and the judge for the warm start."""
    import torch
    from paper_2608_01746_b300 import api, synth, warm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    layers = list(synth.WARM_NET)
    # lab: 32 random objects x 1600 positions = 51,200 training patches from the lab forward
    # model; small: 40 objects x 100 positions
    scales = [("lab", args.warm_objects or 32, args.warm_epochs or 12, 64),
              ("small", 40, 20, 32)]
    results = {}
    clocks = ClockSampler(local)
    clocks.start()
    for name, nobj, epochs, batch in scales:
        cfg = synth.CONFIGS[name]
        t0 = time.perf_counter()
        X, T = warm.training_set(cfg, seeds=range(50000, 50000 + nobj), device=dev)
        torch.cuda.synchronize(dev)
        gen_s = time.perf_counter() - t0
        net = api.wsnet_create(layers, in_side=cfg.N // 2, max_batch=batch, seed=3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        hist = warm.train(net, X, T, epochs, batch, 1e-3, log_every=20)
        e1.record()
        torch.cuda.synchronize(dev)
        train_ms = e0.elapsed_time(e1)
        steps = epochs * (X.shape[0] // batch)
        train_tflops = 3 * warm_flops_per_sample(layers, cfg.N // 2) * steps * batch / (train_ms / 1e3) / 1e12
        sc = synth.make_scan_torch(cfg, device=dev)
        params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
        fused = api.fuse_stack(sc["raw"], cfg.times, params)
        probe = torch.from_numpy(sc["probe"].astype(np.complex64)).to(dev)
        flat = torch.ones((cfg.M, cfg.M), dtype=torch.complex64, device=dev)
        mask = illuminated_mask(sc["probe"], sc["pos"], cfg.M)
        runs = {}
        for start in ("warm", "flat"):
            torch.cuda.synchronize(dev)
            w0 = time.perf_counter()
            if start == "warm":
                ow = warm.warm_object(net, fused, sc["pos"], probe, cfg.M)
                h, chosen, errs = warm.judged_start(fused, sc["pos"], probe, ow, flat, probe_update_start=10 ** 9)
                done = 1
            else:
                h = api.ptycho_init(fused, sc["pos"], flat, probe, probe_update_start=10 ** 9)
                chosen, errs, done = "flat", None, 0
            torch.cuda.synchronize(dev)
            t_s = time.perf_counter() - w0
            obj = np.empty((cfg.M, cfg.M), np.complex64)
            traj = []
            chunk = 5
            while done < 100:
                w0 = time.perf_counter()
                api.ptycho_iterate(h, chunk, errors=False)
                torch.cuda.synchronize(dev)
                t_s += time.perf_counter() - w0
                done += chunk
                api.ptycho_get_object(h, obj)
                traj.append((done, t_s, nrmse_host(obj, sc["obj"], mask)))
            api.ptycho_destroy(h)
            runs[start] = {"chosen_start": chosen, "judge_first_errors": errs, "traj": traj}
        floor = min(v for r in runs.values() for _, _, v in r["traj"])
        goal = 1e-2 if floor <= 1e-2 else 1.05 * floor
        entry = {"train_objects": nobj, "train_patches": int(X.shape[0]), "epochs": epochs, "batch": batch,
                 "data_gen_s": round(gen_s, 2), "train_s": round(train_ms / 1e3, 2),
                 "train_samples_per_s": round(steps * batch / (train_ms / 1e3), 1),
                 "train_tflops": round(train_tflops, 2), "loss_per_epoch": [round(v, 5) for v in hist],
                 "goal_nrmse": round(goal, 5), "floor": round(floor, 5)}
        for start, r in runs.items():
            hit = next(((it, t) for it, t, v in r["traj"] if v <= goal), (None, None))
            entry[start] = {"iterations_to_goal": hit[0], "seconds_to_goal": None if hit[1] is None else round(hit[1], 4),
                            "chosen_start": r["chosen_start"],
                            "judge_first_errors": r["judge_first_errors"],
                            "nrmse_every_5": [round(v, 4) for _, _, v in r["traj"][:12]]}
        results[name] = entry
        api.wsnet_destroy(net)
        del X, T
    clk = clocks.stop()
    lab = results["lab"]
    value = lab["warm"]["seconds_to_goal"]
    out = {"metric": "seconds to the NRMSE goal from the warm start (lab scan)", "value": value, "unit": "s",
           "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16 network (f32 accumulate), f32 reconstruction",
           "data": "synthetic (random objects through the forward model; workload scan held out)",
           "config": {"workload": "learned warm start: 8-layer conv encoder-decoder (2.05 M weights), trained on "
                                  "fused patterns of random objects, prediction stitched into the initial object; "
                                  "lab scan (1024^2 / 256^2 / 1600 positions) and small scan (256^2 / 64^2 / 100)",
                      "probe": "true probe, fixed", "iterations_max": 100},
           "scales": results, "clocks": clk, "e2e": None, "cpu_baseline": None, "roofline": None}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import torch
    from paper_2608_01746_b300 import api, synth

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.CONFIGS[args.workload]
    n_iter = args.iters or cfg.n_iter
    if args.positions:
        import dataclasses
        cfg = dataclasses.replace(cfg, J=args.positions)
    sc = synth.make_scan_torch(cfg, seed=rank_seed(synth.seed_for(args.workload), rank), device=dev)
    raw = sc["raw"]
    J, K, N = raw.shape[0], cfg.K, cfg.N
    M = cfg.M
    params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
    obj0 = torch.ones((M, M), dtype=torch.complex64, device=dev)
    probe0 = torch.from_numpy(sc["probe"].astype(np.complex64)).to(dev)
    pos = sc["pos"]
    fused = torch.empty((J, N, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    stage_ms = np.zeros(4)
    stage_n = np.zeros(4, dtype=np.int64)

    def step(timing=False):
        api.fuse_stack(raw, cfg.times, params, out=fused, stream=stream)
        h = api.ptycho_init(fused, pos, obj0, probe0, stream=stream, fft_path=args.fft)
        if timing:
            api.ptycho_set_timing(h, True)
        api.ptycho_iterate(h, n_iter, errors=False)
        if timing:
            ms, n = api.ptycho_stage_times(h)
            stage_ms[:] += ms
            stage_n[:] += n
        api.ptycho_destroy(h)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(timing=True)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    ms_step = ms_total / args.steps
    updates = J * n_iter * args.steps * world
    value = updates / (ms_total / 1e3)

    # end to end through the same calls with host buffers: H2D of the raw stack, object and
    # probe each step, D2H of the reconstructed object and probe.  Streamed as a pipeline of
    # scans: the raw stack of step k + 1 is copied and fused (fuse_stack_host) on a second
    # stream while step k iterates, and every copy and read-back is inside the timed region.
    e2e = None
    if not args.no_e2e:
        raw_h = raw.cpu().pin_memory()
        obj_h = np.ones((M, M), np.complex64)
        probe_h = sc["probe"].astype(np.complex64)
        out_o = np.empty((M, M), np.complex64)
        out_p = np.empty(probe_h.shape, np.complex64)
        streams = [stream, torch.cuda.Stream(device=dev)]
        raw_d = [torch.empty_like(raw), torch.empty_like(raw)]
        fused_d = [fused, torch.empty_like(fused)]

        def e2e_run(nsteps):
            api.fuse_stack_host(raw_h, raw_d[0], cfg.times, params, out=fused_d[0], stream=streams[0])
            for s in range(nsteps):
                a = s % 2
                h = api.ptycho_init(fused_d[a], pos, obj_h, probe_h, stream=streams[a], fft_path=args.fft)
                api.ptycho_iterate(h, n_iter, errors=False)
                if s + 1 < nsteps:        # the next scan's copy and fusion under this scan's iterations
                    b = 1 - a
                    api.fuse_stack_host(raw_h, raw_d[b], cfg.times, params, out=fused_d[b], stream=streams[b])
                api.ptycho_get_object(h, out_o)
                api.ptycho_get_probe(h, out_p)
                api.ptycho_destroy(h)

        e2e_run(1)
        torch.cuda.synchronize()
        barrier()
        w0 = time.perf_counter()
        e2e_run(args.steps)
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - w0, dist, dev)
        e2e = {"value": updates / e2e_s, "unit": METRIC,
               "h2d_bytes_per_step": int(raw_h.numel() * 2 + obj_h.nbytes + probe_h.nbytes + pos.nbytes),
               "d2h_bytes_per_step": int(out_o.nbytes + out_p.nbytes),
               "pipeline": "scan k + 1's raw stack is copied and fused on a second stream while scan k iterates"}

    # Roofline of the dominant kernel (the exit wave), from the per-stage CUDA events of the timed
    # steps (recorded on the library's stream).  HBM: the kernel's algorithmic bytes per position
    # (A_j, object patch, probe, psi_j': 28 N^2) against the measured copy bandwidth; ALU: its
    # FFT and pointwise flops against the FP32 FMA rate measured by the library's own kernel;
    # iteration: the whole iteration's 36 N^2 bytes per position-update over its time.
    hbm_peak, peak_kind = peaks()
    dom = int(np.argmax(stage_ms))
    names = ["k_exit_wave", "object update (k_object_gather + k_apply)",
             "probe update (k_probe_partial + k_probe_reduce + k_apply)",
             "error (formed in block 0 of the object step's k_apply; empty stage)"]
    Q = cfg.modes
    # the exit-wave stage per iteration: one launch over all J positions, or (N = 256, split last
    # round) the whole-round launch plus the cooperative tail launch; with modes the forward,
    # modulus and inverse launches
    n_timed = args.steps * n_iter
    exit_ms = float(stage_ms[0]) / n_timed
    exit_launches = float(stage_n[0]) / n_timed
    iter_ms = float(stage_ms.sum()) / (args.steps * n_iter)
    fma = api.measure_fp32_fma_tflops(device=dev)
    flops = Q * exit_wave_flops_per_position(N) * J / (exit_ms / 1e3) / 1e12
    hbm_algo = Q * exit_wave_bytes_per_position(N) * J / (exit_ms / 1e3) / 1e9
    traffic = None
    if N == 256 and Q == 1 and EXIT_TRAFFIC["bytes_per_position"] and \
            EXIT_TRAFFIC["sources_sha16"] == exit_kernel_sources_sha16():
        traffic = int(EXIT_TRAFFIC["bytes_per_position"] * J)
    kname = ("k_exit_wave_tma" if N == 256 else ("k_exit_wave128" if N == 128 else "k_exit_wave")) + (
        " (forward + k_modulus_modes + inverse, per iteration)" if Q > 1 else "")
    it_gbs = Q * iteration_bytes_per_update(N) * J / (iter_ms / 1e3) / 1e9
    it_tflops = Q * iteration_flops_per_update(N) * J / (iter_ms / 1e3) / 1e12
    roof = {"kernel": kname, "bound": "hbm",
            "achieved": round(hbm_algo, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(hbm_algo / hbm_peak, 4), "peak_kind": peak_kind,
            "bytes_per_position": exit_wave_bytes_per_position(N), "positions_per_iteration": J,
            "traffic": traffic,
            "traffic_note": (f"ncu DRAM bytes per position {EXIT_TRAFFIC['bytes_per_position']} x {J} positions "
                             f"({EXIT_TRAFFIC['capture']})" if traffic else
                             "null: no ncu capture of the current kernel sources"),
            "ms_per_iteration": round(exit_ms, 4),
            "launches_per_iteration": round(exit_launches, 2),
            "launch_note": ("the whole rounds in one launch and the J mod grid leftover positions in a second, "
                            "cooperative launch (several CTAs per position); achieved = J positions' bytes over "
                            "the two launches' time" if exit_launches > 1.5 and Q == 1 else
                            "one launch per iteration" if Q == 1 else
                            "forward, modulus and inverse launches per iteration"),
            "alu_view": {"achieved_tflops": round(flops, 2), "peak_tflops": round(fma["tflops"], 2),
                         "peak_kind": "measured: the library's FP32 FMA kernel, best of 5 launches",
                         "frac": round(flops / fma["tflops"], 4),
                         "flops_per_position": exit_wave_flops_per_position(N),
                         "derived_peak_tflops_2032mhz": round(fp32_peak_tflops(2032.0), 2)},
            "iteration_view": {"ms_per_iteration": round(iter_ms, 4),
                               "bytes_per_position_update": iteration_bytes_per_update(N),
                               "achieved_gbs": round(it_gbs, 1), "peak_gbs": hbm_peak,
                               "frac": round(it_gbs / hbm_peak, 4),
                               "flops_per_position_update": iteration_flops_per_update(N),
                               "achieved_tflops": round(it_tflops, 2),
                               "alu_frac": round(it_tflops / fma["tflops"], 4)}}
    if args.fft == "dftgemm_bf16x3":
        tflops = dftgemm_flops_per_position(N) * J / (exit_ms / 1e3) / 1e12
        bf16_peak, bf16_kind = bf16_peak_tflops()
        kn = "k_exit_wave_tma<16, FULL, tensor cores>" if N == 256 else f"k_dft{N}_gemm<exit>"
        roof = {"kernel": f"{kn} (tcgen05 split-BF16 DFT-GEMM)", "bound": "tensor",
                "achieved": round(tflops, 2), "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": round(tflops / bf16_peak, 4), "peak_kind": bf16_kind,
                "flops_per_position": dftgemm_flops_per_position(N),
                "traffic": None, "ms_per_iteration": round(exit_ms, 4),
                "launches_per_iteration": round(exit_launches, 2),
                "fp32_fft_equivalent_tflops": round(flops, 2),
                "hbm_view": {"achieved_gbs": round(hbm_algo, 1), "peak_gbs": hbm_peak, "peak_kind": peak_kind,
                             "frac": round(hbm_algo / hbm_peak, 4),
                             "bytes_per_position": exit_wave_bytes_per_position(N)},
                "iteration_view": roof["iteration_view"]}
    fuse_n = fuse_launches(cfg.levels)
    launches = int(args.steps * (fuse_n + 2) + stage_n.sum())

    conv = None
    if rank == 0 and not args.no_nrmse and Q == 1 and args.workload in ("wide64", "wide128"):
        fixed = 10 ** 9
        conv = [time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream, 200,
                              probe_update_start=fixed, fft_path=f)
                for f in ("radix_fp32", "dftgemm_bf16x3")]
    elif rank == 0 and not args.no_nrmse and Q == 1:
        # time to NRMSE 1e-2 (else to 1.05 x the floor) per reading of the data: the default MNF
        # (quantiser on), MNF without the quantiser, MNF with the weighted base, the linear SLI
        # comparator, and the noiseless unclipped intensity itself (what AP alone can reach)
        fixed = 10 ** 9
        it = args.nrmse_iters
        conv = [time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream, it,
                              probe_update_start=0),
                time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream, it,
                              probe_update_start=fixed),
                # the harder start: the probe's aperture alone (its modulus, no phase curvature)
                time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0,
                              probe0.abs().to(probe0.dtype), stream, it, probe_update_start=0,
                              probe_label="aperture-only probe (the true probe's modulus)")]
        for fusion in ("mnf_no_quantiser", "mnf_weighted_base", "sli", "ideal"):
            conv.append(time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream,
                                      5 * it if fusion in ("sli", "ideal") else it, chunk=20,
                                      probe_update_start=fixed, fusion=fusion))
        # the regulariser (alpha = 1e-3 x max, a reading) biases the fixed point; with 1e-4 AP on
        # the noiseless intensity is limited by its own convergence (alpha = 0 diverges at the
        # scan edge, where sum_j |P|^2 is tiny)
        conv.append(time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream, 15 * it, chunk=50,
                                  probe_update_start=fixed, fusion="ideal", alpha=1e-4))
        conv.append(time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream, 30, chunk=5,
                                  probe_update_start=fixed, algorithm="epie_colour"))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        cpu = cpu_baseline()

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.fft == "radix_fp32" else "bf16x3 (split) with f32 accumulate",
        "data": ("synthetic (seeded Fermat-spiral scan, Poisson counts, 16-bit clip)" if N == 256 else
                 "synthetic (seeded jittered raster scan, Poisson counts, 12-bit clip)"),
        "config": {"workload": workload_text(args.workload, n_iter),
                   "fft": args.fft,
                   "modes": Q,
                   "positions": J, "exposures": K, "detector": N, "object": M, "levels": cfg.levels,
                   "iterations": n_iter,
                   "l2": f"inputs larger than L2 (raw stack {raw.numel() * 2 / 1e9:.2f} GB per step)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "stage_ms_per_step": {n: round(float(m) / args.steps, 3) for n, m in zip(names, stage_ms)},
        "dominant_stage": names[dom],
        "roofline": roof, "clocks": clk, "gpu_launches": launches, "e2e": e2e,
        "time_to_nrmse": conv,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def workload_text(name: str, n_iter: int) -> str:
    if name == "lab":
        return ("lab-scale MNF + reconstruction: object 1024x1024 c64, probe 256x256, 1600 positions, "
                f"5 exposures (1/4/16/64/256), 6-level pyramid, {n_iter} iterations per step")
    if name == "mixed":
        return ("mixed-state: the lab scan with 8 incoherent probe modes (+-10% bandwidth), modulus per "
                f"mode, {n_iter} iterations per step")
    if name == "wide128":
        return ("wide 128^2-probe scan: object 1024x1024 c64, probe 128x128, 48x48 raster (2304 positions), "
                f"3 exposures (1/10/100), 4-level pyramid, {n_iter} iterations per step")
    return ("wide 64^2-probe scan: object 1024x1024 c64, probe 64x64, 96x96 raster (9216 positions), "
            f"3 exposures (1/10/100), 4-level pyramid, {n_iter} iterations per step")


# ----------------------------------------------------------------------------- convergence
def illuminated_mask(probe, pos, M):
    N = probe.shape[0]
    den = np.zeros((M, M))
    p2 = np.abs(probe) ** 2
    for y, x in pos:
        den[y:y + N, x:x + N] += p2
    return den >= 0.1 * den.max()


def nrmse_host(obj, truth, mask):
    """min over complex c of ||c O - O_true|| / ||O_true|| on the mask (global phase/scale free)."""
    o = obj[mask].astype(np.complex128)
    t = truth[mask]
    c = np.vdot(o, t) / np.vdot(o, o)
    return float(np.linalg.norm(c * o - t) / np.linalg.norm(t))


def time_to_nrmse(api, sc, cfg, raw, params, fused, pos, obj0, probe0, stream, max_iters, chunk=10,
                  target=1e-2, probe_update_start=0, fusion="mnf", algorithm="ap", fft_path="radix_fp32",
                  alpha=1e-3, probe_label="true probe"):
    """FP32 reconstruction of the benchmarked scan from a flat object with the given probe (the
    known probe, or its aperture alone): NRMSE to the ground truth every `chunk` iterations.
    Device time counts the fusion, set-up and iterations (CUDA events), not the NRMSE
    evaluation."""
    import torch
    M = cfg.M
    mask = illuminated_mask(sc["probe"], pos, M)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if fusion == "mnf":
        api.fuse_stack(raw, cfg.times, params, out=fused, stream=stream)
    elif fusion == "mnf_no_quantiser":
        api.fuse_stack(raw, cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip), delta0=0.0),
                       out=fused, stream=stream)
    elif fusion == "mnf_weighted_base":
        api.fuse_stack(raw, cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip), base_mode="weighted"),
                       out=fused, stream=stream)
    elif fusion == "ideal":
        fused.copy_(sc["intensity"])        # noiseless, unclipped intensity: the reconstruction alone
    else:
        api.fuse_sli(raw, cfg.times, float(cfg.clip), out=fused, stream=stream)
    h = api.ptycho_init(fused, pos, obj0, probe0, alpha_O=alpha, alpha_P=alpha, probe_update_start=probe_update_start,
                        stream=stream, algorithm=algorithm, fft_path=fft_path)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    traj = []
    obj = np.empty((M, M), np.complex64)
    done = 0
    while done < max_iters:
        e0.record(stream)
        api.ptycho_iterate(h, chunk, errors=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms += e0.elapsed_time(e1)
        done += chunk
        api.ptycho_get_object(h, obj)
        traj.append((done, round(t_ms, 2), nrmse_host(obj, sc["obj"], mask)))
    api.ptycho_destroy(h)
    floor = min(v for _, _, v in traj)
    goal = target if floor <= target else 1.05 * floor
    hit = next((it, ms) for it, ms, v in traj if v <= goal)
    every = max(1, len(traj) // 40)
    return {"engine": algorithm, "fft": fft_path, "fusion": fusion, "alpha": alpha, "target": target,
            "reached_target": floor <= target,
            "floor": round(floor, 5), "floor_at_iteration": next(it for it, _, v in traj if v == floor),
            "still_falling": traj[-1][2] <= floor * (1 + 1e-4),
            "goal_used": round(goal, 5), "iterations": hit[0],
            "seconds": round(hit[1] / 1e3, 4),
            "start": f"flat object, {probe_label}, " + ("probe updates on" if probe_update_start == 0
                                                         else "probe fixed"),
            f"trajectory_every_{chunk * every}": [round(v, 5) for _, _, v in traj[every - 1::every]]}


# ----------------------------------------------------------------------------- oracle arm
# The FP64 oracle timed on the host cores: as it stands on one core, and with its per-position
# steps (exit_wave_update, mnf_position) spread over every core by a spawn process pool (the
# object and probe updates stay in the parent, as the oracle writes them).  Amplitudes and the
# exit waves go through shared memory; only the object and probe travel with each task.
_W = {}


def _pool_init(a_name, a_shape, psi_name, psi_shape):
    from multiprocessing import shared_memory
    _W["a_shm"] = shared_memory.SharedMemory(name=a_name)
    _W["A"] = np.ndarray(a_shape, dtype=np.float64, buffer=_W["a_shm"].buf)
    _W["p_shm"] = shared_memory.SharedMemory(name=psi_name)
    _W["psi"] = np.ndarray(psi_shape, dtype=np.complex128, buffer=_W["p_shm"].buf)


def _pool_exit_waves(task):
    import oracle
    obj, probe, pos, js = task
    err = 0.0
    for j in js:
        _W["psi"][j], e = oracle.exit_wave_update(obj, probe, pos[j], _W["A"][j])
        err += e
    return err


def _pool_fuse(task):
    import oracle
    raw, times, kw = task
    p = oracle.FuseParams(**kw)
    return [oracle.mnf_position(r, times, p) for r in raw]


class OraclePool:
    """A spawn pool of `workers` processes over one scan's amplitudes (None: run in-process)."""

    def __init__(self, A, workers: int):
        self.workers = workers
        self.A = A
        self.pool = None
        if workers > 1:
            import multiprocessing as mp
            from multiprocessing import shared_memory
            J, N, _ = A.shape
            self.a_shm = shared_memory.SharedMemory(create=True, size=A.nbytes)
            np.ndarray(A.shape, dtype=np.float64, buffer=self.a_shm.buf)[:] = A
            self.p_shm = shared_memory.SharedMemory(create=True, size=J * N * N * 16)
            self.psi = np.ndarray((J, N, N), dtype=np.complex128, buffer=self.p_shm.buf)
            self.pool = mp.get_context("spawn").Pool(
                workers, initializer=_pool_init, initargs=(self.a_shm.name, A.shape, self.p_shm.name, (J, N, N)))

    def iteration(self, obj, probe, pos):
        """One full-batch iteration, the steps of oracle.iterate_once (object, then probe)."""
        import oracle
        if self.pool is None:
            return oracle.iterate_once(obj, probe, pos, self.A, 1e-3, 1e-3, True)
        chunks = np.array_split(np.arange(len(pos)), self.workers)
        err = sum(self.pool.map(_pool_exit_waves, [(obj, probe, pos, c) for c in chunks]))
        obj = oracle.object_update(obj, probe, pos, self.psi, 1e-3)
        probe = oracle.probe_update(obj, probe, pos, self.psi, 1e-3)
        return obj, probe, err

    def fuse(self, raw, times, p):
        import dataclasses
        import oracle
        if self.pool is None:
            return [oracle.mnf_position(r, times, p) for r in raw]
        chunks = np.array_split(np.arange(len(raw)), self.workers)
        kw = dataclasses.asdict(p)
        out = self.pool.map(_pool_fuse, [(raw[c], times, kw) for c in chunks if len(c)])
        return [x for part in out for x in part]

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.a_shm.close()
            self.a_shm.unlink()
            self.p_shm.close()
            self.p_shm.unlink()


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def lab_oracle_inputs(n_fuse: int):
    import oracle
    from paper_2608_01746_b300 import synth
    cfg = synth.CONFIGS[WORKLOAD]
    sc = synth.make_scan(cfg, frames_for=list(range(n_fuse)))
    A = oracle.amplitudes(sc["intensity"])     # fusing all 1600 positions in FP64 takes ~2 min per core
    return cfg, sc, A


def time_lab_sample(cfg, sc, A, workers: int, n_fuse: int):
    """Per step: fusion of n_fuse positions (the share of one iteration when fusing all J
    positions is amortised over the 200 iterations: J / 200 = 8) and one full-batch iteration
    over all positions.  Returns (seconds, position-updates, fusion seconds)."""
    import oracle
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    obj = np.ones((cfg.M, cfg.M), complex)
    pool = OraclePool(A, workers)
    try:
        pool.fuse(sc["raw"][:1], sc["times"], p)              # workers up and warm
        t0 = time.perf_counter()
        pool.fuse(sc["raw"][:n_fuse], sc["times"], p)
        t1 = time.perf_counter()
        pool.iteration(obj, sc["probe"], sc["pos"])
        t2 = time.perf_counter()
    finally:
        pool.close()
    return t2 - t0, len(sc["pos"]), t1 - t0


def time_small_full(workers: int):
    """The small workload in full: fusion of all 100 positions and 50 iterations."""
    import oracle
    from paper_2608_01746_b300 import synth
    cfg = synth.CONFIGS["small"]
    sc = synth.make_scan(cfg)
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    pool = OraclePool(np.zeros((len(sc["pos"]), cfg.N, cfg.N)), workers)
    try:
        pool.fuse(sc["raw"][:1], sc["times"], p)
        t0 = time.perf_counter()
        fused = np.stack(pool.fuse(sc["raw"], sc["times"], p))
        A = oracle.amplitudes(fused)
        if pool.pool is not None:
            np.ndarray(A.shape, dtype=np.float64, buffer=pool.a_shm.buf)[:] = A
        pool.A = A
        t1 = time.perf_counter()
        obj, probe = np.ones((cfg.M, cfg.M), complex), sc["probe"].astype(complex)
        for _ in range(cfg.n_iter):
            obj, probe, _e = pool.iteration(obj, probe, sc["pos"])
        t2 = time.perf_counter()
    finally:
        pool.close()
    return {"seconds": round(t2 - t0, 2), "fusion_seconds": round(t1 - t0, 3),
            "position_updates_per_s": round(len(sc["pos"]) * cfg.n_iter / (t2 - t0), 1)}


def cpu_baseline():
    """The oracle on one core and on every host core (bounded samples; ~30 s in all)."""
    cores = os.cpu_count() or 1
    n_fuse = 8
    cfg, sc, A = lab_oracle_inputs(max(n_fuse, 8 * cores))
    s1, upd, f1 = time_lab_sample(cfg, sc, A, 1, n_fuse)
    sn, _, _ = time_lab_sample(cfg, sc, A, cores, n_fuse)
    # fusion alone, positions per second (lab frames: 5 x 256^2, 6 levels)
    import oracle
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    pool = OraclePool(A[:1], cores)
    try:
        pool.fuse(sc["raw"][:1], sc["times"], p)
        t0 = time.perf_counter()
        pool.fuse(sc["raw"][:8 * cores], sc["times"], p)
        fn = time.perf_counter() - t0
    finally:
        pool.close()
    return {"value": round(upd / sn, 2), "unit": METRIC, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"FP64 numpy oracle on all {cores} host cores (spawn pool over positions): fusion of "
                       f"{n_fuse} positions + one full-batch iteration over all {upd} positions of the lab scan"),
            "seconds": round(sn, 2),
            "single_core": {"value": round(upd / s1, 2), "seconds": round(s1, 2)},
            "fusion_positions_per_s": {"1_core": round(n_fuse / f1, 2), f"{cores}_cores": round(8 * cores / fn, 2)},
            "small_workload_in_full": {"workload": "small scan: fusion of 100 positions + 50 iterations",
                                       "1_core": time_small_full(1), f"{cores}_cores": time_small_full(cores)}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    n_fuse = 8
    cfg, sc, A = lab_oracle_inputs(n_fuse)
    for _ in range(args.warmup):
        time_lab_sample(cfg, sc, A, cores, 1)
    total = 0.0
    upd = 0
    for _ in range(args.steps):
        dt, u, _f = time_lab_sample(cfg, sc, A, cores, n_fuse)
        total += dt
        upd += u
    value = upd / total
    sample = (f"per step: fusion of {n_fuse} positions + one full-batch iteration over all 1600 positions, "
              f"FP64 numpy oracle on all {cores} host cores")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lab-scale sample: fuse 8 positions + 1 iteration over 1600 positions "
                                   "(object 1024x1024, probe 256x256, 5 exposures, 6 levels)"},
            "cpu_baseline": {"value": round(value, 2), "kind": "oracle", "cores": cores, "cpu_model": cpu_model(),
                             "sample": sample},
            "e2e": {"value": round(value, 2), "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    if args.workload == "warm":
        run_warm(args, world, rank, local)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
