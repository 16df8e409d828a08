"""Benchmark: Image-GS fit steps on a 2048x2048 RGB target with 100k Gaussians.

One step = preprocess/bin + fused forward/L1/adjoint + Adam (the whole hot
path), replayed from a captured CUDA graph. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank fits its own image (independent problems,
no collective on the data path: weak scaling); the max time over ranks is
reported and `value` counts the steps of all ranks.
"""
import argparse
import json
import multiprocessing
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="fit2048_rgb", H=2048, W=2048, n=3, N=100_000, n_sin=8, n_rect=200,
                noise=3, seed=0)
FIT_WORKLOADS = {
    "fit2048_rgb": WORKLOAD,
    "fit256_rgb": dict(name="fit256_rgb", H=256, W=256, n=3, N=4096, n_sin=8, n_rect=20,
                       noise=0, seed=0),
    "fit4096_tex9": dict(name="fit4096_tex9", H=4096, W=4096, n=9, N=500_000, n_sin=8,
                         n_rect=200, noise=3, seed=0),
}
METRIC = "Gaussian-pixel evals/s and fit steps/s (fwd+bwd) vs FP32/SFU roofline"
UNIT = "fit steps/s"
SM_COUNT = 148
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0
# DRAM bytes (read + write) of one fused forward + L1 + adjoint launch of the
# current kernel on the 2048^2 RGB state the bench measures by default (20
# steps from the initial parameters), from one ncu capture of that launch:
# dram__bytes_read.sum 61,402,880 + dram__bytes_write.sum 1,032,704
# (profiles/k_render_fit2048_rgb.md has the command)
FUSED_TRAFFIC_2048_RGB = 62_435_584
TRAFFIC_STEPS_MAX = 50
# library kernels of one fit step (the ncu launch list of the bench):
# preprocess, 2 wide-Gaussian passes, 3 scan passes (the last also writes the
# tile ranges and the evaluation count), emit, the sort of long lists, fused
# adjoint, Adam (whose last CTA also advances the step and writes the loss)
KERNELS_PER_FIT_STEP = 10
# the SSIM term adds the forward render and the one-pass image loss
SSIM_EXTRA_KERNELS = 2


def fused_kernel_ops(evals, pixels, K, n):
    """Algorithmic FP32 lane-ops of one fused forward + L1 + adjoint launch.

    per Gaussian-pixel eval: 2 FADD (d) + 3 FMUL + 2 FFMA (q) + 1 compare = 8
    per pixel, forward blend: K * (3 + n) + n   (shift, scale, Z add, n FMA; 1/Z scaling)
    per pixel, L1 + adjoint: 3n + K * (32 + 3n) (dL/dq, chain rule to 5 params,
                             n colour grads, 5+n reduction adds)
    """
    return evals * 8 + pixels * (K * (3 + n) + n + 3 * n + K * (32 + 3 * n))


def fused_kernel_mufu(pixels, K):
    """Algorithmic special-function operations of one fused launch: per pixel
    K exponentials (the winners' weights) and one reciprocal (1/Z)."""
    return pixels * (K + 1)


class ClockSampler:
    """Samples the SM clock and the throttle reasons while running: through
    NVML (every 20 ms) where the library is present, else nvidia-smi (every
    50 ms plus the query's own time). Read-only queries."""

    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []   # (sm_mhz, sm_max_mhz, set of active reasons)
        self._stop = threading.Event()
        self._t = None
        self._nvml = None
        try:
            import pynvml
            pynvml.nvmlInit()
            self._h = pynvml.nvmlDeviceGetHandleByIndex(index)
            self._nvml = pynvml
            self._bits = {"hw_slowdown": pynvml.nvmlClocksEventReasonHwSlowdown,
                          "hw_thermal_slowdown": pynvml.nvmlClocksEventReasonHwThermalSlowdown,
                          "sw_thermal_slowdown": pynvml.nvmlClocksEventReasonSwThermalSlowdown,
                          "sw_power_cap": pynvml.nvmlClocksEventReasonSwPowerCap}
        except Exception:
            self._nvml = None

    def _sample_nvml(self):
        n = self._nvml
        sm = float(n.nvmlDeviceGetClockInfo(self._h, n.NVML_CLOCK_SM))
        mx = float(n.nvmlDeviceGetMaxClockInfo(self._h, n.NVML_CLOCK_SM))
        r = n.nvmlDeviceGetCurrentClocksEventReasons(self._h)
        self.samples.append((sm, mx, {k for k, b in self._bits.items() if r & b}))

    def _sample_smi(self):
        out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                              "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=5).stdout.strip()
        if out:
            f = [x.strip() for x in out.split(",")]
            sm = float(f[0]) if f[0].replace(".", "").isdigit() else None
            mx = float(f[1]) if f[1].replace(".", "").isdigit() else None
            self.samples.append((sm, mx, {self.REASONS[i] for i in range(4)
                                          if len(f) > 3 + i and f[3 + i].lower() == "active"}))

    def _run(self):
        while not self._stop.is_set():
            try:
                self._sample_nvml() if self._nvml else self._sample_smi()
            except Exception:
                pass
            self._stop.wait(0.02 if self._nvml else 0.05)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [x[0] for x in self.samples if x[0] is not None]
        mx = [x[1] for x in self.samples if x[1] is not None]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = sorted(set().union(*[x[2] for x in self.samples]))
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples),
                "via": "nvml" if self._nvml else "nvidia-smi"}


def rank_env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_workload(w, rank):
    """Each rank fits its own image: the same workload drawn with seed + rank."""
    return dict(w, seed=w["seed"] + rank)


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's mean step time; every rank must call it."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms, world):
    """Whole-job steps per second: every rank completes one step per `ms`."""
    return world * 1000.0 / ms


def make_inputs(w=WORKLOAD):
    from paper_2407_01866_b300 import synth
    if w["n"] == 9:   # albedo RGB, normal XYZ in [-1, 1], roughness, metallic, AO
        target = synth.texture_stack(w["H"], w["W"], seed=w["seed"], n_sin=w["n_sin"],
                                     n_rect=w["n_rect"], noise_octaves=w["noise"])
        lo = [0, 0, 0, -1, -1, -1, 0, 0, 0]
        d = synth.gaussians(w["N"], 9, seed=w["seed"], color_lo=lo, color_hi=1.0)
    else:
        target = synth.target_image(w["H"], w["W"], w["n"], seed=w["seed"], n_sin=w["n_sin"],
                                    n_rect=w["n_rect"], noise_octaves=w["noise"])
        d = synth.gaussians(w["N"], w["n"], seed=w["seed"])
    return target, synth.packed(d)


def host_cores():
    """(cores this process may run on, os.cpu_count())."""
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count() or 1
    return usable, os.cpu_count()


def _oracle_worker(job):
    """One oracle process: forward + L1 sign + adjoint, 16 pixels at a time,
    over pixels[start::stride] until the deadline. Returns pixels done."""
    P, target_sample, pix, H, W, n, start, stride, deadline = job
    from oracle import image_gs as O
    g = O.Gaussians.from_packed(P)
    done = 0
    mine = pix[start::stride]
    tgt = target_sample[start::stride]
    for c0 in range(0, len(mine), 16):
        if time.time() > deadline:
            break
        chunk = mine[c0:c0 + 16]
        pts = O.pixel_centres(chunk)
        img = O.render_points(g, pts, H, W)
        go = np.sign(img - tgt[c0:c0 + 16]) / (H * W * n)
        O.backward_points(g, pts, go, H, W)
        done += len(chunk)
    return done


def cpu_baseline(target, P, budget_s=15.0, seed=0, w=WORKLOAD):
    """The oracle's fit step (forward + L1 + adjoint, float64 brute force over
    all N Gaussians per pixel) on random pixels of the workload, one process
    per usable host core for about budget_s seconds, extrapolated to the
    frame."""
    from paper_2407_01866_b300 import synth
    H, W, n = w["H"], w["W"], w["n"]
    usable, total = host_cores()
    pix = synth.sample_pixels(64 * usable + 4096, H, W, seed=seed)
    tsample = target[:, pix[:, 0], pix[:, 1]].T.copy()
    # one thread per process: the processes are the parallelism
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = multiprocessing.get_context("spawn")   # never fork a CUDA process
        with ctx.Pool(usable) as pool:
            pool.map(_oracle_worker, [(P, tsample[:16], pix[:16], H, W, n, 0, 1,
                                       time.time() + 60.0)] * usable)   # imports, warm-up
            t0 = time.time()
            jobs = [(P, tsample, pix, H, W, n, r, usable, t0 + budget_s) for r in range(usable)]
            done = sum(pool.map(_oracle_worker, jobs))
            dt = time.time() - t0
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    step_s = dt / max(done, 1) * H * W
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": usable, "kind": "oracle",
            "host_cpu_count": total,
            "sample": f"{done} random pixels of the {H}x{W} workload in {dt:.1f} s on {usable} "
                      f"processes (affinity mask of {usable} of {total} host cores), "
                      f"forward + L1 + adjoint brute force in float64 over all {w['N']} "
                      "Gaussians, extrapolated to the full frame"}


def run_reference(args):
    rank = rank_env()[1]
    if rank != 0:
        return
    target, P = make_inputs()
    times = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(target, P, budget_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)),
                          seed=i)
        if i >= args.warmup:
            times.append(1.0 / cb["value"])
    ms = 1000.0 * statistics.mean(times)
    v = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "H": 2048, "W": 2048, "n": 3,
                       "N": 100_000, "K": 10, "tile": 16},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "host_cpu_count": cb["host_cpu_count"], "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args, w=WORKLOAD):
    import torch
    from paper_2407_01866_b300 import lib as L

    world, rank, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W, n, N = w["H"], w["W"], w["n"], w["N"]
    target_np, P_np = make_inputs(rank_workload(w, rank))
    cfg = L.default_config(ssim_weight=args.ssim)
    target = torch.from_numpy(target_np).to(dev)
    P0 = torch.from_numpy(P_np).to(dev)

    # size the intersection capacity from the initial binning, with headroom
    binner = L.Binner(N, n, H, W, cfg)
    bins0 = binner.bin(L.packed_view(P0, n))
    st0 = L.read_stats(bins0)
    cap = int(st0.m_needed * 3) + 4096
    ws = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, cap), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2

    # the dominant kernel (fused forward + L1 + adjoint) on the initial parameters
    evals_init = int(st0.evals)
    k_ms_init = None
    if not args.kernel_once:
        G0 = torch.zeros_like(P0)
        view0 = L.packed_view(P0, n)
        k_ms_init = _time_events(lambda: L.render_backward(view0, bins0, cfg, None, target, G0),
                                 20, flush, warmup=3)
        del G0
    del binner, bins0

    P = P0.clone()
    G = torch.zeros_like(P)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    step = torch.zeros(1, dtype=torch.int32, device=dev)
    state = L.FitState(P.data_ptr(), G.data_ptr(), m.data_ptr(), v.data_ptr(), step.data_ptr(),
                       N, n)
    loss = torch.zeros(1, device=dev)

    # Sec. 4.1 half-precision storage: float32 master, half copy rendered
    half = None
    if args.storage != "f32":
        half = torch.zeros(P.shape, dtype={"f16": torch.float16, "bf16": torch.bfloat16}[
            args.storage], device=dev)

    def step_fn(stream=None):
        if half is None:
            L.fit_step(state, target, H, W, cfg, ws, cap, loss, stream=stream)
        else:
            L.fit_step_half(state, half, target, H, W, cfg, ws, cap, loss, stream=stream)

    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step_fn(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_fn()

    if args.kernel_once:
        # the fit (graph replays, as timed below), then one binning, one forward
        # and one fused adjoint launch on the fitted state (for ncu captures)
        for _ in range(args.steps):
            graph.replay()
        torch.cuda.synchronize()
        bins = L.preprocess_bin(L.packed_view(P, n), H, W, cfg, ws, cap)
        img = torch.empty((n, H, W), device=dev)
        L.render_forward(bins, cfg, img)
        L.render_backward(L.packed_view(P, n), bins, cfg, None, target, G)
        torch.cuda.synchronize()
        return

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: K graph replays, L2 flushed between steps ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            starts[i].record()
            graph.replay()
            ends[i].record()
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        ms = float(statistics.mean(step_ms))
        ms = max_over_ranks(ms, dist, dev)
        if dist:
            dist.barrier()

        # binning statistics of the final state (evals of one forward)
        stats = L.read_stats(L.preprocess_bin(L.packed_view(P, n), H, W, cfg, ws, cap))
        if stats.flags & L.FLAG_CAPACITY:
            raise RuntimeError("intersection capacity exceeded during the benchmark")
        evals = int(stats.evals)
        pixels = H * W

        # ---- dominant kernel (fused forward + L1 + adjoint), timed alone on
        # the final state, on the stream it is launched on ----
        bins = L.preprocess_bin(L.packed_view(P, n), H, W, cfg, ws, cap)
        view = L.packed_view(P, n)
        k_ms = _time_events(lambda: L.render_backward(view, bins, cfg, None, target, G), 20,
                            flush, warmup=3)

        # ---- measured peaks of this GPU: FP32 FMA lanes and the exp2 unit ----
        from paper_2407_01866_b300 import peaks
        fp32_peak = max(peaks.probe("ffma", iters=2000, reps=5)[0],
                        peaks.probe("ffma2", iters=1000, reps=5)[0])
        mufu_peak = peaks.probe("ex2", iters=500, reps=5)[0]
    ops = fused_kernel_ops(evals, pixels, cfg.K, n)
    achieved = ops / (k_ms * 1e-3)
    mufu_ops = fused_kernel_mufu(pixels, cfg.K)
    ops_init = fused_kernel_ops(evals_init, pixels, cfg.K, n)

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its target from pinned host memory and reads its loss
    # back. Two device target buffers, each with its own captured step: the
    # copy for step k+1 (on a copy stream) overlaps step k.
    # the pinned copy is filled through its numpy view: host-to-device copies
    # from pinned pages written that way measured 55 GB/s, against 17-27 GB/s
    # after torch's own CPU copy or fill into the same pages
    tgt_host = torch.empty(target_np.shape, dtype=torch.float32, pin_memory=True)
    tgt_host.numpy()[...] = target_np
    loss_host = torch.zeros(1).pin_memory()
    e_steps = max(3, min(args.steps, 50))
    targets = [target, torch.empty_like(target)]
    graphs = [graph, torch.cuda.CUDAGraph()]
    target_now = target
    with torch.cuda.graph(graphs[1]):
        target = targets[1]
        step_fn()
    target = target_now
    # the second graph's first replay uploads it: once, untimed, on a real target
    targets[1].copy_(target)
    graphs[1].replay()
    cs = torch.cuda.Stream(device=dev)
    comp = torch.cuda.current_stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    cs.wait_stream(comp)
    with torch.cuda.stream(cs):
        targets[0].copy_(tgt_host, non_blocking=True)
        copied[0].record(cs)
    for k in range(e_steps):
        b = k & 1
        if k + 1 < e_steps:  # next step's input, once its buffer's last user is done
            with torch.cuda.stream(cs):
                if k >= 1:
                    cs.wait_event(used[1 - b])
                targets[1 - b].copy_(tgt_host, non_blocking=True)
                copied[1 - b].record(cs)
        comp.wait_event(copied[b])
        graphs[b].replay()
        used[b].record(comp)
        loss_host.copy_(loss, non_blocking=True)
    comp.wait_stream(cs)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e_steps

    if rank == 0:
        value = job_throughput(ms, world)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if half is None else f"f32 math, {args.storage} parameter storage",
            "data": "synthetic",
            "config": {"workload": w["name"], "H": H, "W": W, "n": n, "N": N, "K": cfg.K,
                       "storage": args.storage, "loss": ("L1" if args.ssim == 0 else
                                                         f"L1 + {args.ssim} SSIM"),
                       "bits_per_pixel": N * (5 + n) * (32 if half is None else 16) / (H * W),
                       "tile": cfg.tile, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"independent fits x{world}"},
            "gaussian_pixel_evals_per_step": evals,
            "gaussian_pixel_evals_per_s": world * evals * 1000.0 / ms,
            "final_loss": float(loss.item()),
            "gpu_launches": (KERNELS_PER_FIT_STEP + (0 if half is None else 2)
                             + (SSIM_EXTRA_KERNELS if args.ssim > 0 else 0)) * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
                         "unit": "T fp32 lane-ops/s", "frac": achieved / fp32_peak,
                         "traffic": (FUSED_TRAFFIC_2048_RGB
                                     if w["name"] == "fit2048_rgb" and half is None
                                     and args.steps <= TRAFFIC_STEPS_MAX else None),
                         "traffic_unit": "bytes per launch",
                         "traffic_state": ("ncu DRAM read + write of this kernel after 20 fit "
                                           "steps from the initial parameters; reported for "
                                           f"runs of at most {TRAFFIC_STEPS_MAX} steps"),
                         "kernel": "k_render_bwd (fused forward + L1 + adjoint)",
                         "kernel_ms": k_ms, "ops_per_launch": ops,
                         "peak_note": "measured on this GPU in this run (libigs_peaks: chains of "
                                      "fma.rn.f32 and fma.rn.f32x2 over every SM, the faster "
                                      "lane rate), under the clocks reported below; "
                                      f"nominal {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x "
                                      f"{SM_MAX_MHZ:.0f} MHz = "
                                      f"{SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ / 1e6:.1f} T",
                         "mufu": {"ops_per_launch": mufu_ops, "peak": mufu_peak / 1e12,
                                  "unit": "T ex2/s (measured)",
                                  "frac": mufu_ops / (k_ms * 1e-3) / mufu_peak},
                         "initial_state": {"kernel_ms": k_ms_init, "evals": evals_init,
                                           "ops_per_launch": ops_init,
                                           "achieved": ops_init / (k_ms_init * 1e-3) / 1e12,
                                           "frac": ops_init / (k_ms_init * 1e-3) / fp32_peak}},
            "e2e": {"value": world * 1000.0 / e2e_ms, "unit": UNIT,
                    "h2d_bytes_per_step": int(target.numel() * 4), "d2h_bytes_per_step": 4},
            "clocks": clocks.summary(),
        }
        if not args.no_cpu_baseline and world == 1:   # the oracle baseline runs at N = 1 only
            line["cpu_baseline"] = cpu_baseline(target_np, P_np, budget_s=args.cpu_budget, w=w)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def _time_events(fn, steps, flush=None, warmup=0):
    """Mean ms of fn() over `steps` runs (after `warmup` untimed ones), CUDA
    events on the current stream, L2 flushed before each run if given."""
    import torch
    for i in range(warmup):
        if flush is not None:
            flush.fill_(i & 0xff)
        fn()
    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.fill_(i & 0xff)
        st[i].record()
        fn()
        en[i].record()
    torch.cuda.synchronize()
    return float(statistics.mean(a.elapsed_time(b) for a, b in zip(st, en)))


def run_batch(args):
    """64 images, sides log-uniform in 256-2048, one Gaussian per 28 px: batched
    persistent fit step (autotuned mapping) vs 64 single-image fit steps, both
    replayed from CUDA graphs."""
    import torch
    from paper_2407_01866_b300 import lib as L
    from paper_2407_01866_b300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    shapes = synth.batch_shapes(64, seed=0)
    Hs = [h for h, _, _ in shapes]
    Ws = [w for _, w, _ in shapes]
    Ns = [m for _, _, m in shapes]
    n = 3
    cfg = L.default_config()
    Ps = [synth.packed(synth.gaussians(N, n, seed=b)) for b, N in enumerate(Ns)]
    Ts = [synth.target_image(H, W, n, seed=100 + b, n_rect=20) for b, (H, W) in
          enumerate(zip(Hs, Ws))]
    P_all = torch.from_numpy(np.concatenate(Ps)).to(dev)
    T_all = torch.from_numpy(np.concatenate([t.ravel() for t in Ts])).to(dev)

    def state(P):
        G, m, v = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
        step = torch.zeros(1, dtype=torch.int32, device=dev)
        keep = (P, G, m, v, step)
        s_ = L.FitState(P.data_ptr(), G.data_ptr(), m.data_ptr(), v.data_ptr(),
                        step.data_ptr(), P.shape[0], n)
        s_._keep = keep
        return s_

    shape = L.batch_shape(Hs, Ws, Ns, n)
    cap = 12 * sum(Ns) + 4096
    ws = L.alloc_workspace(L.batch_workspace_size(shape, cfg, cap), dev)
    L.batch_setup(shape, cfg, ws, cap)
    Pb = P_all.clone()
    sb = state(Pb)
    loss_b = torch.zeros(64, device=dev)
    tuning, tune_ms = L.autotune_batch(sb, T_all, shape, cfg, ws, cap, reps=3)

    def capture(fn):
        s_ = torch.cuda.Stream(device=dev)
        s_.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s_):
            fn()
        torch.cuda.current_stream().wait_stream(s_)
        g_ = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_):
            fn()
        return g_

    gb = capture(lambda: L.fit_batch_step(sb, T_all, shape, cfg, ws, cap, tuning=tuning,
                                          loss_out=loss_b))
    # sequential: one plain fit step per image, all 64 in one graph
    seq = []
    off_p, off_t = 0, 0
    for b in range(64):
        N, H, W = Ns[b], Hs[b], Ws[b]
        Pi = P_all[off_p:off_p + N].clone()
        ti = T_all[off_t:off_t + n * H * W]
        c = 12 * N + 1024
        wsi = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, c), dev)
        seq.append((state(Pi), ti, H, W, wsi, c, torch.zeros(1, device=dev)))
        off_p += N
        off_t += n * H * W

    def seq_step():
        for si, ti, H, W, wsi, c, li in seq:
            L.fit_step(si, ti, H, W, cfg, wsi, c, li)

    gs = capture(seq_step)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        gb.replay()
        gs.replay()
    torch.cuda.synchronize()
    steps = min(args.steps, 100)
    with ClockSampler(0) as clocks:
        ms_b = _time_events(gb.replay, steps, flush)
        ms_s = _time_events(gs.replay, steps, flush)
    px = sum(h * w for h, w in zip(Hs, Ws))
    line = {"metric": "images x fit steps/s (batched persistent form vs 64 sequential plain "
                      "fit steps)", "value": 64 * 1000.0 / ms_b, "unit": "image-steps/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch64", "images": 64, "pixels": px, "gaussians": sum(Ns),
                       "sides": "log-uniform 256-2048", "K": cfg.K, "tile": cfg.tile,
                       "l2": "flushed between timed steps (256 MB write)"},
            "tuning": {"ctas_per_sm": tuning.ctas_per_sm, "stage": tuning.stage,
                       "order": tuning.order, "adjoint_ms": tune_ms},
            "sequential": {"value": 64 * 1000.0 / ms_s, "ms_per_step": ms_s},
            "speedup_vs_sequential": ms_s / ms_b,
            "clocks": clocks.summary()}
    print(json.dumps(line))


def run_decode(args):
    """8192x8192 RGB, 2M Gaussians: full-frame render and 1M random-point decode
    with parameters stored as float32, float16 and bfloat16."""
    import torch
    from paper_2407_01866_b300 import lib as L
    from paper_2407_01866_b300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    c = synth.CONFIGS["decode8192_rgb"]
    H, W, n, N, Q = c["H"], c["W"], c["n"], c["N"], c["Q"]
    d = synth.gaussians(N, n, seed=0)
    pts = torch.from_numpy(synth.query_points(Q, H, W, seed=0)).to(dev)
    cfg = L.default_config()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    img = torch.empty((n, H, W), device=dev)
    out = torch.empty((Q, n), device=dev)
    res = {}
    steps = min(args.steps, 50)
    with ClockSampler(0) as clocks:
        for name, dt in (("f32", torch.float32), ("f16", torch.float16), ("bf16", torch.bfloat16)):
            ts = [torch.from_numpy(d[k]).to(dev).to(dt) for k in ("xy", "theta", "inv_scale",
                                                                  "color")]
            view = L.gaussians_view(*ts)
            binner = L.Binner(N, n, H, W, cfg, m_capacity=8 * N)
            bins = binner.bin(view)
            st = L.read_stats(bins)
            cap = binner.m_capacity
            for _ in range(args.warmup):
                L.preprocess_bin(view, H, W, cfg, binner.ws, cap)
                L.render_forward(bins, cfg, img)
                L.decode_points(bins, cfg, pts, out)
            ms_bin = _time_events(lambda: L.preprocess_bin(view, H, W, cfg, binner.ws, cap),
                                  steps, flush)
            ms_fwd = _time_events(lambda: L.render_forward(bins, cfg, img), steps, flush)
            ms_dec = _time_events(lambda: L.decode_points(bins, cfg, pts, out), steps, flush)
            res[name] = {"bin_ms": ms_bin, "render_ms": ms_fwd, "frame_evals": int(st.evals),
                         "render_evals_per_s": st.evals / (ms_fwd * 1e-3),
                         "decode_ms": ms_dec, "queries_per_s": Q / (ms_dec * 1e-3),
                         "param_bytes": sum(t.numel() * t.element_size() for t in ts)}
    line = {"metric": "full-frame Gaussian-pixel evals/s and random-point queries/s by "
                      "parameter storage", "value": res["f16"]["queries_per_s"],
            "unit": "queries/s (f16 storage)", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": res["f16"]["decode_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 math, f16/bf16/f32 storage", "data": "synthetic",
            "config": {"workload": "decode8192", "H": H, "W": W, "n": n, "N": N, "queries": Q,
                       "l2": "flushed between timed launches (256 MB write)"},
            "by_storage": res,
            "half_vs_f32": {k: {"decode_speedup": res["f32"]["decode_ms"] / res[k]["decode_ms"],
                                "render_speedup": res["f32"]["render_ms"] / res[k]["render_ms"],
                                "render_evals_per_s_ratio": res[k]["render_evals_per_s"]
                                / res["f32"]["render_evals_per_s"]}
                            for k in ("f16", "bf16")},
            "clocks": clocks.summary()}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--workload", default="fit2048_rgb",
                    choices=list(FIT_WORKLOADS) + ["batch64", "decode8192"])
    ap.add_argument("--ssim", type=float, default=0.0,
                    help="weight of the SSIM term of the fit loss (Sec. 4.1 uses 0.1; "
                         "0 = L1 with the fused adjoint)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="parameter storage of the fit workloads (f16/bf16: half copy "
                         "rendered, float32 master updated)")
    ap.add_argument("--kernel-once", action="store_true",
                    help="run the fit for --steps steps, then bin, render and run the fused "
                         "adjoint once on the fitted state and exit (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "decode8192":
        run_decode(args)
    else:
        run_ours(args, FIT_WORKLOADS[args.workload])


if __name__ == "__main__":
    main()
