#!/usr/bin/env python
"""Benchmark of the free-flight expansion on GB300: realizations per second.

One step = the whole hot path on one batch of the workload: the per-axis
passes of eq. FF (pre-chirp, FFT, k-space phase, fold or inverse FFT with the
post-chirp and term sum) along every axis, then |Psibar|^2 -- every kernel of
``ffx_expand``.  Inputs are seeded synthetic fields (see
paper_1602_03395_gb300/inputs.py) resident in HBM when the timed region
starts; successive steps read distinct realizations from a pool larger than
L2.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ffx|reference]
                  [--workload large_two_cloud|large_quasicondensate|two_cloud|1d|
                   quasicondensate|mixed] [--form auto|paper|fold|dense|tc]
                  [--unsplit] [--batch B] [--column AXIS] [--no-cpu-baseline]
                  [--no-companion]

The default workload is the largest single-GPU configuration: the 256^3
two-cloud interferometer at lam = 100, t = 400, one realization per step; the
line also carries the same measurement of the 128x128x1024 quasicondensate at
lam = 100 as an extra record (``extra_records``).

Multi-GPU (torchrun, one rank per GPU): realizations are independent, so each
rank expands its own share with no collective on the data path (weak
scaling); only the timing is reduced (max over ranks).

``--impl reference`` times the FP64 CPU oracle (oracle/) on the host cores on
the same workload and prints the same line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1602_03395_gb300 import inputs  # noqa: E402

METRIC = "realizations/s and HBM GB/s vs peak at rel-L2 density err <=2e-5 vs FP64"
E2E_MAX_LANES = 4  # end-to-end leg: streams (each with its own plan) steps alternate over
UNIT = "realizations/s"
L2_BYTES = 129 * 1024 * 1024
SMS, FP32_LANES = 152, 128


# ---------------------------------------------------------------------------
# multi-rank host logic (one process per GPU): disjoint seeded shards, the
# slowest rank's time, the whole job's rate
# ---------------------------------------------------------------------------

def rank_realizations(rank: int, batch: int, n_buffers: int = 4):
    """First realization index of each of a rank's distinct input buffers of
    `batch` realizations: rank r draws [(1000 r + i) B, (1000 r + i + 1) B),
    disjoint across ranks."""
    return [(rank * 1000 + i) * batch for i in range(n_buffers)]


def mixed_seed(rank: int, i: int) -> int:
    """Seed of instance i of the mixed batch on rank `rank` (disjoint across
    ranks for batches below 7919 instances)."""
    return rank * 7919 + i


def max_over_ranks(torch, dist, value: float, device) -> float:
    """The largest of the ranks' values (the slowest rank's time)."""
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps: int, per_rank: int, world: int, ms: float) -> float:
    """Whole-job realizations/s: every rank ran `steps` steps of `per_rank`
    realizations in (at most) `ms` milliseconds."""
    return steps * per_rank * world / (ms * 1e-3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ffx", choices=["ffx", "reference"])
    ap.add_argument("--workload", default="large_two_cloud",
                    choices=["two_cloud", "1d", "quasicondensate", "large_two_cloud",
                             "large_quasicondensate", "mixed"])
    ap.add_argument("--form", default="auto", choices=["auto", "paper", "fold", "dense", "tc"])
    ap.add_argument("--unsplit", action="store_true",
                    help="with --form tc: one TF32 product on rounded operands (reported variant, "
                         "density error of order 1e-3)")
    ap.add_argument("--bf16", action="store_true",
                    help="BF16 operands on the streaming tensor-core passes (kind::f16; split into heads and "
                         "tails, or unsplit with --unsplit); the automatic form's default")
    ap.add_argument("--tf32", action="store_true",
                    help="split TF32 operands on every tensor-core pass (the automatic form's BF16 default off)")
    ap.add_argument("--batch", type=int, default=None, help="realizations per step (default: workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-backward", action="store_true",
                    help="skip the ffx_expand_backward record of the workload")
    ap.add_argument("--fft-passes", action="store_true",
                    help="time the FFT-form (fold) passes at lam = 1 and 2 on 64^3 x 64, 256^3 and 1-D N=1024 x 65536 "
                         "lines, per pass against the HBM roofline (one JSON line)")
    ap.add_argument("--no-companion", action="store_true",
                    help="large_two_cloud: skip the 128x128x1024 quasicondensate extra record")
    ap.add_argument("--column", type=int, default=None, metavar="AXIS",
                    help="output the detector image: the density integrated along AXIS (Sec. 6)")
    args = ap.parse_args()
    if args.unsplit and (args.form != "tc" or args.workload == "mixed"):
        ap.error("--unsplit needs --form tc and a single-lattice workload")
    if args.bf16 and (args.form not in ("auto", "tc") or args.workload == "mixed"):
        ap.error("--bf16 needs --form auto or tc and a single-lattice workload")
    if args.tf32 and args.bf16:
        ap.error("--tf32 and --bf16 exclude each other")
    return args


def workload(name, batch):
    w = inputs.WORKLOADS[name]()
    w.key = name  # the command-line name (keys of the committed traffic records)
    if batch is not None:
        w.batch = batch
    return w


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def pass_flops(N: int, lam: int, lines: int, form: str) -> float:
    """Algorithmic FP32 flops of one axis pass (5 N log2 N per complex FFT of
    length N; 6 per complex multiply, 2 per complex add).
    paper form, per term: FFT + IFFT + pre-chirp, k-phase, post-chirp
    multiplies + accumulate = 10 N log2 N + 20 N.
    dense form: the per-axis map as an N x N complex matrix, 8 N per point.
    fold form, per term: FFT + pre-chirp and k-phase multiplies + fold add
    = 5 N log2 N + 14 N; plus one inverse FFT per line."""
    lg = math.log2(N)
    if form == "paper":
        return lines * lam * (10 * N * lg + 20 * N)
    if form in ("dense", "tc"):
        return lines * 8.0 * N * N  # N x N complex matrix times each line
    return lines * (lam * (5 * N * lg + 14 * N) + 5 * N * lg)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def cpu_oracle_rate(w, psi=None, budget_s=12.0):
    """The FP64 oracle on the host cores: realizations/s over a bounded sample
    (psi: realizations already drawn, else four are drawn)."""
    import oracle as O
    if psi is None:
        psi = [w.realization(r) for r in range(4)]
    O.expand_density(psi[0], w.dx, w.t, w.lam)  # warm
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or n == 0:
        O.expand_density(psi[n % len(psi)], w.dx, w.t, w.lam)
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args):
    """FP64 CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.workload, args.batch)
    import oracle as O
    n_pool = 4 if w.batch * int(np.prod(w.dims)) <= 1 << 22 else 2
    pool = [w.batch_array(w.batch, start=i * w.batch) for i in range(n_pool)]
    for i in range(args.warmup):
        O.expand_density(pool[i % n_pool], w.dx, w.t, w.lam)
    t0 = time.perf_counter()
    for i in range(args.steps):
        O.expand_density(pool[i % n_pool], w.dx, w.t, w.lam)
    dt = time.perf_counter() - t0
    value = args.steps * w.batch / dt
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "dims": list(w.dims), "dx": list(w.dx), "lam": list(w.lam),
                   "t": w.t, "batch": w.batch},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps x {w.batch} realization(s) of {w.name}, "
                                   "FP64 per-axis dense maps via BLAS on all host cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# comparison baselines (timed only; never on the product path): the same
# per-axis recipe of eq. FF with every fine index q batched into one library
# FFT call per axis -- cuFFT through torch.fft on the GPU, pocketfft through
# scipy.fft on the host cores (FFTW is not installed here)
# ---------------------------------------------------------------------------

def recipe_tables(N, lam, dx, t):
    """Phase factors of eqs. presA, presB, presf (paper form) for one axis,
    default offsets (a = -L/2, abar centring the magnified box), FP64."""
    L = N * dx
    s = -(((lam - 1) * N) // 2)
    tau = math.pi * t / (L * L)
    q = np.arange(lam, dtype=np.float64)[:, None]
    n = np.arange(N, dtype=np.float64)[None, :]
    m = np.arange(N)
    l = np.where(2 * m < N, m, m - N).astype(np.float64)[None, :]
    P = np.exp(-2j * np.pi * np.mod(q * n, lam * N) / (lam * N))
    K = np.exp(2j * np.pi * (l * s / N - tau * l * l - (2 * tau / lam) * l * q))
    F = np.exp(2j * np.pi * (q * s / (lam * N) + q * n / N - tau * q * q / lam ** 2)) / lam
    nii = np.mod(lam * np.arange(N), N)
    return P, K, F, nii


def recipe_axis_torch(torch, x, axis, tabs):
    """One axis of the paper-form recipe with torch.fft (cuFFT) on a [B, ...] field."""
    P, K, F, nii = tabs
    x = x.movedim(axis, -1)
    y = torch.fft.fft(x.unsqueeze(0) * P.view((P.shape[0],) + (1,) * (x.dim() - 1) + (P.shape[1],)), dim=-1)
    y = torch.fft.ifft(y * K.view((K.shape[0],) + (1,) * (x.dim() - 1) + (K.shape[1],)), dim=-1)
    y = (y[..., nii] * F.view((F.shape[0],) + (1,) * (x.dim() - 1) + (F.shape[1],))).sum(0)
    return y.movedim(-1, axis)


def cufft_baseline(torch, w, dev, steps=20):
    """Realizations/s of the same recipe on cuFFT (torch.fft), complex64."""
    tabs = []
    for N, lam, dx in zip(w.dims, w.lam, w.dx):
        P, K, F, nii = recipe_tables(N, lam, dx, w.t)
        tabs.append((torch.from_numpy(P.astype(np.complex64)).to(dev),
                     torch.from_numpy(K.astype(np.complex64)).to(dev),
                     torch.from_numpy(F.astype(np.complex64)).to(dev), torch.from_numpy(nii).to(dev)))
    x = torch.from_numpy(w.batch_array(w.batch)).to(dev)

    def run():
        y = x
        for j in range(len(w.dims)):
            y = recipe_axis_torch(torch, y, 1 + j, tabs[j])
        return (y.abs() ** 2)

    try:
        out = run()
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        return {"value": w.batch / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                "kind": "same per-axis recipe (paper form, all q batched) on cuFFT via torch.fft, complex64",
                "result": out}
    except RuntimeError as exc:  # e.g. out of memory for lam * M intermediates
        return {"value": None, "unit": UNIT, "kind": "cuFFT recipe", "error": str(exc)[:200]}


def scipy_baseline(w, budget_s=8.0, dtype=np.complex64):
    """Realizations/s of the same recipe with scipy.fft (pocketfft) on all host cores."""
    import scipy.fft as sfft
    workers = os.cpu_count()
    tabs = [recipe_tables(N, lam, dx, w.t) for N, lam, dx in zip(w.dims, w.lam, w.dx)]
    tabs = [(P.astype(dtype), K.astype(dtype), F.astype(dtype), nii) for P, K, F, nii in tabs]
    x0 = w.realization(0).astype(dtype)[None]

    def run(x):
        for j, (P, K, F, nii) in enumerate(tabs):
            y = np.moveaxis(x, 1 + j, -1)
            sh = (P.shape[0],) + (1,) * (y.ndim - 1) + (P.shape[1],)
            y = sfft.fft(y[None] * P.reshape(sh), axis=-1, workers=workers)
            y = sfft.ifft(y * K.reshape(sh), axis=-1, workers=workers)
            y = (y[..., nii] * F.reshape(sh)).sum(0)
            x = np.moveaxis(y, -1, 1 + j)
        return np.abs(x) ** 2

    run(x0)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or n == 0:
        run(x0)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": workers,
            "kind": f"same per-axis recipe on scipy.fft (pocketfft), {np.dtype(dtype).name}",
            "sample": f"{n} realizations in {dt:.1f} s"}


def pipelined_e2e(torch, dev, plans, call, h_in, d_in, d_out, h_out, steps):
    """End-to-end milliseconds for `steps` steps, each copying its input from
    pinned host memory (h_in[i % len(h_in)]), expanding it through the C ABI
    and copying the densities back to pinned host memory.  Steps alternate
    between len(plans) lanes (stream, plan, device and host buffers), so that
    one lane's copies overlap the others' expansions, as a streaming caller
    runs it; every step still moves its own bytes both ways."""
    main = torch.cuda.current_stream(dev)
    lanes = [torch.cuda.Stream(dev) for _ in plans]
    for k, st in enumerate(lanes):  # warm each lane
        with torch.cuda.stream(st):
            d_in[k].copy_(h_in[k % len(h_in)], non_blocking=True)
            call(plans[k], d_in[k], d_out[k])
            h_out[k].copy_(d_out[k], non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for st in lanes:
        st.wait_event(e0)
    if len(lanes) == 1:
        with torch.cuda.stream(lanes[0]):
            for i in range(steps):
                d_in[0].copy_(h_in[i % len(h_in)], non_blocking=True)
                call(plans[0], d_in[0], d_out[0])
                h_out[0].copy_(d_out[0], non_blocking=True)
    else:
        for i in range(steps):
            k = i % len(lanes)
            with torch.cuda.stream(lanes[k]):
                d_in[k].copy_(h_in[i % len(h_in)], non_blocking=True)
                call(plans[k], d_in[k], d_out[k])
                h_out[k].copy_(d_out[k], non_blocking=True)
    for st in lanes:
        main.wait_stream(st)
    e1.record(main)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def host_api_e2e(torch, dev, ffx, plans, h_in, h_out, steps):
    """End-to-end milliseconds for `steps` steps of ffx_expand_host (one C
    call per step: pinned host input -> device -> expansion -> pinned host
    densities), alternating between len(plans) lanes (stream, plan and host
    output buffer each), so that one lane's copies overlap the others'
    expansions."""
    main = torch.cuda.current_stream(dev)
    lanes = [torch.cuda.Stream(dev) for _ in plans]
    for k, st in enumerate(lanes):  # warm each lane (the plan's staging buffers)
        ffx.ffx_expand_host(plans[k], h_in[k % len(h_in)], h_out[k], stream=st)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for st in lanes:
        st.wait_event(e0)
    n = len(lanes)
    for i in range(steps):
        k = i % n
        ffx.ffx_expand_host(plans[k], h_in[i % len(h_in)], h_out[k], stream=lanes[k])
    for st in lanes:
        main.wait_stream(st)
    e1.record(main)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def load_traffic(kernel_key: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the kernel's current sources (the files the
    record names); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    from paper_1602_03395_gb300 import build as B
    entry = rec.get(kernel_key)
    if not entry or not entry.get("sources"):
        return None
    try:
        if entry.get("sources_digest") != B.sources_digest(entry["sources"]):
            return None
    except OSError:
        return None
    return entry.get("bytes_per_launch")


def mixed_flops(specs, form, bf16=False):
    """Algorithmic flops of one call: (all, the share on BF16 operands).  With
    BF16 phases every pass of a tensor-core plan (lines of 32 to 256 points,
    a multiple of 16) runs on the BF16 kernel."""
    tot = bf = 0.0
    for dims, dx, t, lam in specs:
        M = int(np.prod(dims))
        for j, N in enumerate(dims):
            f = pass_flops(N, lam[j], M // N, form)
            tot += f
            if bf16 and 32 <= N <= 256 and N % 16 == 0:
                bf += f
    return tot, bf


def mixed_backward_record(args, torch, ffx, plan, ws, x, stream):
    """ffx_expand_backward on the mixed-batch plan (every instance's gradient
    with respect to psi0 for a seeded normal dL/drho), CUDA events over direct
    calls after warm-up; the rel-L2 error of the first instance's gradient
    against the FP64 oracle's."""
    g = torch.from_numpy(np.random.default_rng(12).normal(size=plan.points).astype(np.float32)).to(x.device)
    out = torch.empty_like(x)
    for _ in range(3):
        ffx.ffx_expand_backward(plan, x, g, out)
    torch.cuda.synchronize()
    n0 = plan.launch_count()
    ffx.ffx_expand_backward(plan, x, g, out)
    per_call = plan.launch_count() - n0
    steps = max(3, min(args.steps, 20))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ffx.ffx_expand_backward(plan, x, g, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    import oracle as O
    w = ws[0]
    m = int(np.prod(w.dims))
    psi = x[:m].cpu().numpy().reshape((1,) + tuple(w.dims))
    gi = g[:m].cpu().numpy().reshape((1,) + tuple(w.dims))
    ref = O.density_loss_gradient(psi, gi, w.dx, w.t, w.lam)
    got = out[:m].cpu().numpy().reshape(ref.shape)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"value": len(ws) / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms, "calls": steps,
            "gpu_launches_per_call": per_call, "rel_l2_grad_err_vs_fp64_first_instance": err,
            "loss": "dL/drho a seeded normal field",
            "timing": "CUDA events around direct calls on the stream"}


def run_mixed(args, torch, dist, world, rank, dev):
    """The mixed-lattice ensemble: every instance of the batch in one
    ffx_expand on a many-instance plan (one persistent kernel per axis pass,
    replayed as a CUDA graph)."""
    from paper_1602_03395_gb300 import ffx
    count = args.batch or 1000
    ws = inputs.config_mixed_batch(count=count)
    specs = [(w.dims, w.dx, w.t, w.lam) for w in ws]
    plan = ffx.PlanMany(specs, form=args.form, tf32=args.tf32)
    # a few distinct realizations per lattice shape, repeated to fill the batch
    # (the values do not change the work; all instances stay distinct buffers)
    cache = {}
    x = torch.empty(plan.points, dtype=torch.complex64, device=dev)
    views = plan.unpack(x)
    for i, w in enumerate(ws):
        key = (tuple(w.dims), i % 3)
        if key not in cache:
            cache[key] = torch.from_numpy(w.realization(mixed_seed(rank, i))).to(dev)
        views[i].copy_(cache[key])
    out = torch.empty(plan.points, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # parity of this configuration against the FP64 oracle (rank 0): the first
    # instance of every lattice shape, from the same packed call
    err = None
    if rank == 0:
        import oracle as O
        ffx.ffx_expand(plan, x, out)
        torch.cuda.synchronize()
        seen = set()
        err = {}
        for i, w in enumerate(ws):
            if tuple(w.dims) in seen:
                continue
            seen.add(tuple(w.dims))
            m, off = int(np.prod(w.dims)), plan.offsets[i]
            psi = x[off:off + m].cpu().numpy().reshape((1,) + tuple(w.dims))
            ref = O.expand_density(psi, w.dx, w.t, w.lam)[0]
            got = out[off:off + m].cpu().numpy().reshape(w.dims)
            err["x".join(map(str, w.dims)) + f"_lam{w.lam[0]}"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    for _ in range(args.warmup):
        ffx.ffx_expand(plan, x, out)
    n0 = plan.launch_count()
    ffx.ffx_expand(plan, x, out)
    per_call = plan.launch_count() - n0  # the call's graph: one kernel per phase
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ffx.ffx_expand(plan, x, out)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        ms = max_over_ranks(torch, dist, ms, dev)
    value = job_rate(args.steps, count, world, ms)
    flops, flops_bf = mixed_flops(specs, plan.form, plan.bf16)
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    alu_peak = SMS * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (ms / args.steps * 1e-3) / 1e12
    if plan.form == "tc":
        # tensor-core phases: `achieved` counts the algorithmic 8 N flops per
        # point; the peak is that of the call's mix, the flops on BF16 operands
        # at the BF16 peak and the rest at the TF32 peak (time-weighted:
        # all flops / (bf16 flops / P_bf16 + tf32 flops / P_tf32))
        tf_peak, tf_src = tensor_peak(pk, pk_src, ms)
        bf_peak, bf_src = tensor_peak(pk, pk_src, ms, "bf16")
        tc_peak = flops / (flops_bf / bf_peak + (flops - flops_bf) / tf_peak)
        kern = ("dense_bf16_many_kernel<false> (per-thread copies) and <true> (TMA tiles)" if plan.bf16
                else "dense_tc_kernel<false, true, false>")
        roofline = {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": achieved / tc_peak,
                    "traffic": load_traffic(f"many_tc_mixed_{count}_call" + ("_bf16" if plan.bf16 else "")),
                    "kernel": kern + " (all phases of one call)",
                    "executed_tflops": 3 * achieved, "bf16_flop_share": flops_bf / flops,
                    "peak_source": (f"BF16 share at {bf_src}; the rest at {tf_src}" if plan.bf16 else tf_src)}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak,
                    "traffic": load_traffic(f"many_dense_mixed_{count}_call") if plan.form == "dense" else None,
                    "kernel": ("many_dense_kernel" if plan.form == "dense" else "many_kernel") + " (all phases of one call)",
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({pk_src})"}
    byts = sum(int(np.prod(d)) * (8 + 16 * (len(d) - 1) + 4) for d, _, _, _ in specs)
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    # end to end: pinned host input -> expand -> pinned host densities, two lanes
    hx = x.cpu().pin_memory()
    plan2 = ffx.PlanMany(specs, form=args.form, tf32=args.tf32)
    steps_e2e = max(2, min(args.steps, 20))
    e2e_ms = host_api_e2e(torch, dev, ffx, [plan, plan2], [hx],
                          [torch.empty(plan.points, dtype=torch.float32).pin_memory() for _ in range(2)], steps_e2e)
    lanes_used = 2
    plan2.close()
    if world > 1:
        e2e_ms = max_over_ranks(torch, dist, e2e_ms, dev)
    backward = None
    if rank == 0 and not args.no_backward:
        backward = mixed_backward_record(args, torch, ffx, plan, ws, x, stream)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"mixed_{count}_instances_48^3_64^3_96^3_128x32x32_lam10-100",
                       "batch_per_gpu": count, "form": plan.form, "points_per_step": plan.points,
                       "precision": ("split BF16 on the tensor cores (kind::f16, three products)" if plan.bf16 else
                                     "split TF32 on the tensor cores (three products)" if plan.form == "tc"
                                     else "FP32"),
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs {plan.points * 8 / 2**30:.2f} GiB > 129 MB L2"},
            "rel_l2_density_err_vs_fp64": err,
            "gpu_launches": per_call * args.steps,
            "clocks": clocks,
            "roofline": roofline,
            "roofline_hbm": {"bound": "hbm", "achieved": byts / (ms / args.steps * 1e-3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": byts / (ms / args.steps * 1e-3) / 1e9 / hbm_peak},
            "e2e": {"value": job_rate(steps_e2e, count, world, e2e_ms), "unit": UNIT, "api": "ffx_expand_host",
                    "lanes": lanes_used,
                    "h2d_bytes_per_step": plan.points * 8, "d2h_bytes_per_step": plan.points * 4},
            "cpu_baseline": None,
            "backward": backward,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def tensor_peak(pk, pk_src, timed_ms, dtype="tf32"):
    """Dense tensor peak for the tensor-core passes: the measured bf16 cuBLAS
    figure -- the burst one for a timed region under a second, the sustained
    one for longer regions -- as it stands for BF16 operands, times the
    nominal TF32 : BF16 dense ratio (1.1 : 2.25 PFLOP/s) for TF32 operands."""
    key = "bf16_tflops" if (timed_ms < 1000.0 or "bf16_tflops_sustained" not in pk) else "bf16_tflops_sustained"
    if dtype == "bf16":
        return float(pk.get(key, 1900.0)), f"{key} (BF16 dense), {pk_src}"
    return (float(pk.get(key, 1900.0)) * 1.1 / 2.25,
            f"{key} x 1.1/2.25 (TF32 dense : BF16 dense, nominal), {pk_src}")


def backward_record(args, torch, ffx, plan, w, pool_in, distinct, stream, M):
    """ffx_expand_backward on the bench's plan for the loss L = sum (rho - tau)^2,
    tau the density of an independent realization: dL/drho = 2 (rho - tau)
    from the FP64 oracle (lattices up to 2^25 points; a seeded normal field
    above), the batch's gradient with respect to psi0 over K calls after W
    warm-up calls (inputs from the rotating pool, so larger than L2), CUDA
    events on the stream; the kernels one call launches; the rel-L2 error of
    the first realization's gradient against the oracle's."""
    B_ = pool_in[0].shape[0]
    shape = tuple(pool_in[0].shape)
    small = M <= 1 << 25 and len(distinct) > 1
    if small:
        import oracle as O
        psi = distinct[0].numpy()[:1]
        rho = O.expand_density(psi, w.dx, w.t, w.lam)
        tau = O.expand_density(distinct[1].numpy()[:1], w.dx, w.t, w.lam)
        g1 = (2.0 * (rho - tau)).astype(np.float32)
        g = torch.from_numpy(np.broadcast_to(g1, shape).copy())
    else:
        g = torch.from_numpy(np.random.default_rng(11).normal(size=shape).astype(np.float32))
    g = g.to(pool_in[0].device)
    out = torch.empty_like(pool_in[0])
    n = len(pool_in)
    for i in range(max(3, args.warmup)):
        ffx.ffx_expand_backward(plan, pool_in[i % n], g, out)
    torch.cuda.synchronize()
    n0 = plan.launch_count()
    ffx.ffx_expand_backward(plan, pool_in[0], g, out)
    per_call = plan.launch_count() - n0
    steps = max(3, min(args.steps, 20))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        ffx.ffx_expand_backward(plan, pool_in[(i + 1) % n], g, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    err = None
    if small:
        got = ffx.ffx_expand_backward(plan, pool_in[0][:1].contiguous(), g[:1].contiguous()).cpu().numpy()
        ref = O.density_loss_gradient(psi, g1, w.dx, w.t, w.lam)
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"value": B_ / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms, "batch": B_, "calls": steps,
            "gpu_launches_per_call": per_call, "rel_l2_grad_err_vs_fp64": err,
            "loss": ("L = sum (rho - tau)^2, tau the density of an independent realization; dL/drho from "
                     "the FP64 oracle" if small else "dL/drho a seeded normal field"),
            "timing": "CUDA events around direct calls on the stream, inputs rotating through the pool"}


def hbm_step_record(w, batch, chain, fused_call, out_bytes, step_ms, hbm_peak, pk_src):
    """Whole-step HBM view: the algorithmic bytes of a step (read psi0, 8 B
    per point, write the output) and the bytes the implementation's launches
    move (the BF16 chain's input split, 16 B per point; every pass one read
    and one write of the batch, 8 + 8 B per point, 4 B for densities; the fused
    launch keeps its intermediates in L2), over the step's time."""
    pts = batch * int(np.prod(w.dims))
    algo = pts * 8 + out_bytes
    if fused_call:
        impl = algo
    else:
        impl = (16 * pts if chain else 0) + (len(w.dims) - 1) * 16 * pts + pts * 8 + out_bytes
    sec = step_ms * 1e-3
    return {"algorithmic_bytes": algo, "implementation_bytes": impl, "unit": "GB/s", "peak": hbm_peak,
            "algorithmic_gbs": algo / sec / 1e9, "algorithmic_frac": algo / sec / 1e9 / hbm_peak,
            "implementation_gbs": impl / sec / 1e9, "implementation_frac": impl / sec / 1e9 / hbm_peak,
            "note": f"per step over ms_per_step; of {pk_src} hbm_gbs"}


def precision_label(args, bf16, chain=False):
    op = "BF16" if bf16 else "TF32"
    if args.unsplit:
        return f"{op} unsplit: one product on rounded operands (reported variant; density error of order 1e-3)"
    if bf16:
        return (("BF16 chain: the input split into BF16 head and tail planes, every pass on them "
                 "(kind::f16, three products), planes between the passes; " if chain else
                 "split BF16 on the streaming tensor-core passes (kind::f16, three products); ")
                + "split TF32 on the other tensor-core passes, else FP32")
    return "split TF32 on the tensor cores (three products), else FP32"


def measure_workload(args, torch, dist, world, rank, local, dev, ffx, w, primary=True):
    """One single-lattice workload: the K steps replayed from CUDA graphs and
    timed with CUDA events, per-pass durations from a separate traced graph,
    the error against the FP64 oracle over the whole output, the roofline of
    the dominant launch, and the end-to-end rate through the host-buffer call.
    Returns the JSON record (rank 0) or None."""
    B_ = w.batch
    M = int(np.prod(w.dims))
    plan = ffx.Plan(w.dims, w.dx, w.t, w.lam, form=args.form, unsplit=args.unsplit, bf16=args.bf16,
                    tf32=args.tf32)
    form = plan.form
    order = plan.pass_order()
    fused_call = plan.fused and B_ <= plan.fused_max_batch  # all d passes in one launch
    call_forms = plan.call_forms(B_)  # the kernel each axis runs at this batch
    # BF16 chain: one launch splits the input into BF16 planes, then the passes
    chain = plan.bf16_chain(B_) and args.column is None
    if args.column is None:
        out_shape = (B_,) + tuple(w.dims)

        def call(x, out=None):
            return ffx.ffx_expand(plan, x, out)
    else:
        # detector image: the integrated axis runs last; unfused calls add one
        # (untraced) launch that sums the densities along it
        col = args.column
        out_shape = (B_,) + tuple(n for j, n in enumerate(w.dims) if j != col)
        order = [j for j in order if j != col] + [col]

        def call(x, out=None):
            return ffx.ffx_expand_column(plan, x, col, out)

    # input pool larger than L2: distinct buffers, each step reads the next one
    step_in_bytes = B_ * M * 8
    pool_n = max(2, math.ceil(2 * L2_BYTES / step_in_bytes))
    pool_n = min(pool_n, 256)
    n_distinct = 4 if B_ * M <= 1 << 22 else 2  # large lattices: drawing a realization takes seconds
    distinct = [torch.from_numpy(w.batch_array(B_, start=s)) for s in rank_realizations(rank, B_, n_distinct)]
    pool_in = [distinct[i % n_distinct].to(dev) for i in range(pool_n)]
    pool_out = [torch.empty(out_shape, dtype=torch.float32, device=dev) for _ in range(min(pool_n, 64))]
    stream = torch.cuda.current_stream(dev)

    # parity of this very configuration against the FP64 oracle (rank 0, first
    # realization, the whole output lattice)
    err = None
    if rank == 0 and M <= 1 << 25:
        import oracle as O
        if args.column is None:
            ref = O.expand_density(distinct[0].numpy()[:1], w.dx, w.t, w.lam)
        else:
            ref = O.column_density(distinct[0].numpy()[:1], w.dx, w.t, w.lam, args.column)
        got = call(pool_in[0][:1].contiguous()).cpu().numpy()
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        del ref, got

    for i in range(args.warmup):
        call(pool_in[i % pool_n], pool_out[i % len(pool_out)])
    torch.cuda.synchronize()
    # one more call, counted: the kernels it launches (the library's own
    # count) and the traced intervals it records (one per pass; a BF16 chain
    # adds its input split, a pass that splits its own input records both
    # launches in its interval)
    n0 = plan.launch_count()
    trial = [torch.cuda.Event(enable_timing=True) for _ in range(64)]
    plan.trace(trial)
    call(pool_in[0], pool_out[0])
    launches = plan.trace_count() // 2
    plan.trace(None)
    per_call = plan.launch_count() - n0
    torch.cuda.synchronize()

    # The K steps are captured into CUDA graphs of up to GRAPH_STEPS steps and
    # replayed back to back: the device runs the same kernels on the same
    # buffers as K separate calls, without host launch gaps between them.
    # Only these plain graphs run in the timed region.
    GRAPH_STEPS = 200
    chunk = min(args.steps, GRAPH_STEPS)
    graphs = []  # (graph, steps)
    done = 0
    while done < args.steps:
        n = min(chunk, args.steps - done)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for i in range(done, done + n):
                call(pool_in[i % pool_n], pool_out[i % len(pool_out)])
        graphs.append((g, n))
        done += n
    # Per-launch durations come from a separate graph of the first steps whose
    # launches carry event-record nodes (the library's trace hook; each adds
    # ~2-4 us), replayed once before the timed region and never inside it.
    TRACED_STEPS = 20
    n_traced = min(TRACED_STEPS, args.steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * launches * n_traced)]
    traced = torch.cuda.CUDAGraph()
    plan.trace(ev)
    with torch.cuda.graph(traced):
        for i in range(n_traced):
            call(pool_in[i % pool_n], pool_out[i % len(pool_out)])
    plan.trace(None)
    for g, _ in graphs:  # warm the graphs
        g.replay()
    traced.replay()
    torch.cuda.synchronize()
    # clocks are sampled over a window of sustained load (>= 0.6 s of the same
    # graphs) that ends with the timed region, so a short timed region still
    # falls inside the sampled window
    sampler = ClockSampler(local)
    sampler.start()
    t_load = time.perf_counter()
    while time.perf_counter() - t_load < 0.6:
        for g, _ in graphs:
            g.replay()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for g, _ in graphs:
        g.replay()
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end)
    if world > 1:
        ms = max_over_ranks(torch, dist, ms, dev)

    # per-pass durations from the traced graph's events
    per_pass = [[] for _ in range(launches)]
    for s in range(n_traced):
        for k in range(launches):
            i0 = 2 * (s * launches + k)
            per_pass[k].append(ev[i0].elapsed_time(ev[i0 + 1]))
    mean_ms = [statistics.mean(v) for v in per_pass]
    launch_time = ("CUDA events around each launch, from a traced graph replayed outside the timed "
                   "region (its event nodes add ~2-4 us per launch)")
    if launches == 1:
        # one launch per step: the step time of the timed (untraced) region is
        # the launch time
        mean_ms = [ms / args.steps]
        launch_time = "one launch per step: the timed region's step time (CUDA events at its ends)"
    # the lattice axis of each traced launch (None: the BF16 split of a chain)
    launch_axis = ([None] if chain else []) + list(order)
    dom = max((k for k in range(launches) if fused_call or launch_axis[k] is not None), key=lambda k: mean_ms[k])
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    alu_peak = SMS * FP32_LANES * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    out_bytes = 4 * int(np.prod(out_shape))
    # operands of the dominant tensor-core launch: BF16 where the plan gives
    # the streaming kernel's passes BF16 (lines of N = 32k >= 64 outside the
    # tensor-memory kernels' 64-point case), else TF32
    dom_axis = order[0] if fused_call else launch_axis[dom]
    bf16_launch = (plan.bf16 and not fused_call and call_forms[dom_axis] == "tc"
                   and w.dims[dom_axis] >= 64 and w.dims[dom_axis] % 32 == 0
                   and not (w.dims[dom_axis] == 64 and B_ * M // 64 <= 4 * 128 * SMS))
    if fused_call:
        # one cooperative launch runs every pass (dense map: FP32 SIMT, or the
        # tensor cores when every axis has 64 points); HBM sees the input read
        # and the output written, the intermediates stay in L2
        fused_tc = call_forms[0] == "tc" and args.column is None  # detector images: the FP32 fused kernel
        axis_form = "tc" if fused_tc else "fused"
        flops = sum(pass_flops(w.dims[j], w.lam[j], B_ * M // w.dims[j], "dense") for j in order)
        kernel_key = f"fused_{'tc' if fused_tc else 'dense'}_{'x'.join(map(str, w.dims))}_{w.key}"
        if args.column is not None:
            kernel_key += f"_column{args.column}"
        traffic = load_traffic(f"{kernel_key}_b{B_}")
        bytes_launch = B_ * M * 8 + out_bytes
        pass_names = ["fused_" + "_".join(f"axis{j}" for j in order)]
    else:
        axis = dom_axis
        N, lam = w.dims[axis], w.lam[axis]
        axis_form = call_forms[axis]
        flops = pass_flops(N, lam, B_ * M // N, axis_form)
        # HBM view of the same launch: it reads and writes the batch once
        # (complex64; the last pass writes float32 densities)
        last = dom == launches - 1
        kernel_key = f"pass_{axis_form}_N{N}_lam{lam}_{w.key}" + ("_bf16" if bf16_launch else "")
        if args.column is not None:
            kernel_key += f"_column{args.column}"
        traffic = load_traffic(f"{kernel_key}_b{B_}" + ("_density" if last else ""))
        bytes_launch = B_ * M * (8 + (4 if last else 8))
        pass_names = ["split_bf16_planes" if j is None else f"axis{j}_N{w.dims[j]}_lam{w.lam[j]}_{call_forms[j]}"
                      for j in launch_axis]
    achieved = flops / (mean_ms[dom] * 1e-3) / 1e12
    if axis_form == "tc":
        # split contraction on the tensor cores; `achieved` counts the
        # algorithmic 8 N^2 flops per line, the tensor cores execute 3x that
        # (three split products)
        tc_peak, tc_src = tensor_peak(pk, pk_src, ms, "bf16" if bf16_launch else "tf32")
        roofline = {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": achieved / tc_peak, "traffic": traffic, "kernel": kernel_key,
                    "launch_ms": mean_ms[dom], "launch_time": launch_time,
                    "executed_tflops": (1 if args.unsplit else 3) * achieved,
                    "peak_source": tc_src}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": traffic,
                    "kernel": kernel_key, "launch_ms": mean_ms[dom], "launch_time": launch_time,
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                   f"(sm_max_mhz from MEASURED_PEAKS.json, {pk_src})"}

    value = job_rate(args.steps, B_, world, ms)

    # end to end through the C ABI with host buffers: pinned H2D, expand, D2H
    # per step, over 1 .. E2E_MAX_LANES lanes (see host_api_e2e); lanes beyond
    # the first have their own plan (staging buffers, workspace) and stream
    lane_plans = [plan] + [ffx.Plan(w.dims, w.dx, w.t, w.lam, form=args.form, unsplit=args.unsplit, bf16=args.bf16,
                                    tf32=args.tf32)
                           for _ in range(E2E_MAX_LANES - 1)]
    if args.column is None:
        def call_pl(pl, x, out):
            return ffx.ffx_expand(pl, x, out)
    else:
        def call_pl(pl, x, out):
            return ffx.ffx_expand_column(pl, x, args.column, out)
    e2e_steps = max(2, min(args.steps, 200))
    h_in = [d.pin_memory() for d in distinct]
    h_out = [torch.empty(out_shape, dtype=torch.float32).pin_memory() for _ in range(E2E_MAX_LANES)]
    # 1 .. E2E_MAX_LANES lanes, the fastest kept: one step alone is a serial chain
    # (input copy, expansion, density copy); more lanes overlap one step's copies
    # with the others' expansions
    if args.column is None:
        # the C ABI's host-buffer call, one per step
        e2e_api = "ffx_expand_host"
        e2e_lanes = {n: host_api_e2e(torch, dev, ffx, lane_plans[:n], h_in, h_out, e2e_steps)
                     for n in range(1, E2E_MAX_LANES + 1)}
    else:
        e2e_api = "torch copies + ffx_expand_column"
        d_in = [torch.empty_like(pool_in[0]) for _ in range(E2E_MAX_LANES)]
        d_out = [torch.empty(out_shape, dtype=torch.float32, device=dev) for _ in range(E2E_MAX_LANES)]
        e2e_lanes = {n: pipelined_e2e(torch, dev, lane_plans[:n], call_pl, h_in, d_in, d_out, h_out, e2e_steps)
                     for n in range(1, E2E_MAX_LANES + 1)}
    lanes_used = min(e2e_lanes, key=e2e_lanes.get)
    e2e_ms = e2e_lanes[lanes_used]
    for pl in lane_plans[1:]:
        pl.close()
    if world > 1:
        e2e_ms = max_over_ranks(torch, dist, e2e_ms, dev)
    e2e_value = job_rate(e2e_steps, B_, world, e2e_ms)

    # the fringe readout of eq. dphase2 on the step's detector image (two-cloud
    # workloads imaged across their separation axis): one launch, timed alone
    fringe = None
    if primary and args.column is not None and w.fringe is not None and w.fringe[0] != args.column:
        sep_axis, D = w.fringe
        img = pool_out[0][0]
        y_dim = [j for j in range(len(w.dims)) if j != args.column].index(sep_axis)
        y0, dy = ffx.output_axis(plan, sep_axis)
        for _ in range(3):
            ph = ffx.ffx_fringe_phase(img, y0, dy, D, w.t, y_dim=y_dim)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(100):
            ffx.ffx_fringe_phase(img, y0, dy, D, w.t, y_dim=y_dim)
        f1.record(stream)
        torch.cuda.synchronize()
        fringe = {"us_per_image": f0.elapsed_time(f1) * 10.0, "rows": int(ph.numel()),
                  "separation_axis": sep_axis, "D": D,
                  "median_phase_rad": float(torch.nanmedian(ph).item())}

    cufft = scipy64 = scipy32 = None
    if primary and rank == 0 and world == 1 and not args.no_cpu_baseline and args.column is None:
        cufft = cufft_baseline(torch, w, dev, steps=20 if B_ * M <= 1 << 22 else 5)
        res = cufft.pop("result", None)
        if res is not None:
            ours = ffx.ffx_expand(plan, pool_in[0].contiguous())
            cufft["max_rel_diff_vs_ffx"] = float(((res - ours).norm() / ours.norm()).item())
            del res, ours
        if M * B_ <= 1 << 22:
            scipy32 = scipy_baseline(w, dtype=np.complex64)
            scipy64 = scipy_baseline(w, dtype=np.complex128)

    # the gradient of an image-space loss (ffx_expand_backward: T^H (2 g . T psi0))
    # on the same plan, timed with CUDA events over direct calls; its error
    # against the FP64 oracle's gradient for the first realization
    backward = None
    if primary and rank == 0 and args.column is None and not args.no_backward:
        backward = backward_record(args, torch, ffx, plan, w, pool_in, distinct, stream, M)

    cpu = None
    if primary and rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, dt = cpu_oracle_rate(w, [d.numpy()[0] for d in distinct])
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} realizations of {w.name} in {dt:.1f} s, FP64 per-axis dense "
                         "maps via BLAS on all host cores"}
    plan.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "dims": list(w.dims), "dx": list(w.dx),
                   "lam": list(w.lam), "t": w.t, "batch_per_gpu": B_, "form": form,
                   "axis_forms": list(plan.axis_forms), "call_forms": list(call_forms),
                   "fused_one_launch": bool(fused_call),
                   "precision": precision_label(args, plan.bf16, chain),
                   "output": ("density" if args.column is None else
                              f"detector image: density integrated along axis {args.column}"),
                   "parallelism": f"replicas x{world} (realizations sharded, no collective)",
                   "l2": f"rotating pool of {pool_n} input buffers "
                         f"({pool_n * step_in_bytes / 2**20:.0f} MiB > 129 MB L2)",
                   "timed_region_ms": ms},
        "rel_l2_density_err_vs_fp64": err,
        "rel_l2_scope": "whole output lattice of the first realization, against the FP64 oracle",
        "gpu_launches": per_call * args.steps,
        "graph": f"K steps replayed as {len(graphs)} CUDA graph(s) of <= {GRAPH_STEPS} steps, no trace "
                 f"nodes; pass_ms from a separate graph of {n_traced} traced steps run before the timed region",
        "clocks": clocks,
        "roofline": roofline,
        "roofline_hbm": {"bound": "hbm", "achieved": bytes_launch / (mean_ms[dom] * 1e-3) / 1e9,
                         "peak": hbm_peak, "unit": "GB/s",
                         "frac": bytes_launch / (mean_ms[dom] * 1e-3) / 1e9 / hbm_peak,
                         "note": f"of {pk_src} hbm_gbs; one read + one write of the batch"},
        "hbm_step": hbm_step_record(w, B_, chain, fused_call, out_bytes, ms / args.steps, hbm_peak, pk_src),
        "pass_ms": {pass_names[k]: mean_ms[k] for k in range(launches)},
        "e2e": {"value": e2e_value, "unit": UNIT, "api": e2e_api, "lanes": lanes_used,
                "h2d_bytes_per_step": B_ * M * 8,
                "d2h_bytes_per_step": out_bytes},
        "cpu_baseline": cpu,
        "backward": backward,
        "fringe_readout": fringe,
        "comparisons": {"cufft_recipe": cufft, "cpu_fft_recipe_c64": scipy32,
                        "cpu_fft_recipe_c128": scipy64},
    }


FFT_PASS_CASES = [
    ("64^3 x 64", (64, 64, 64), 64),
    ("256^3", (256, 256, 256), 1),
    ("1-D N=1024 x 65536", (1024,), 65536),
]


def run_fft_passes(args, torch, dev, ffx):
    """The FFT (fold) form's passes where they move more bytes than they
    compute (lam = 1 and 2): per-pass CUDA events around each launch of a
    traced graph (median of 20 replays), bytes = one read and one write of the
    batch (complex64; the last pass writes float32 densities), against the
    measured HBM copy figure."""
    pk, pk_src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    cases = []
    for name, dims, batch in FFT_PASS_CASES:
        for lam in (1, 2):
            d = len(dims)
            plan = ffx.Plan(dims, (0.25,) * d, 1.0, (lam,) * d, form="fold")
            M = int(np.prod(dims))
            xs = [torch.randn((batch,) + dims, dtype=torch.complex64, device=dev) for _ in range(2)]
            out = torch.empty((batch,) + dims, dtype=torch.float32, device=dev)
            n = plan.launches_per_call(batch=batch)
            for i in range(3):
                ffx.ffx_expand(plan, xs[i % 2], out)
            reps = 20
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n * reps)]
            g = torch.cuda.CUDAGraph()
            plan.trace(ev)
            with torch.cuda.graph(g):
                for i in range(reps):
                    ffx.ffx_expand(plan, xs[i % 2], out)
            plan.trace(None)
            g.replay()
            torch.cuda.synchronize()
            order = plan.pass_order()
            passes = []
            for k in range(n):
                ms = statistics.median(ev[2 * (r * n + k)].elapsed_time(ev[2 * (r * n + k) + 1]) for r in range(reps))
                byts = batch * M * (8 + (4 if k == n - 1 else 8))
                passes.append({"axis": order[k], "N": dims[order[k]], "ms": ms, "bytes": byts,
                               "gbs": byts / (ms * 1e-3) / 1e9, "frac": byts / (ms * 1e-3) / 1e9 / hbm,
                               "out": "density" if k == n - 1 else "complex"})
            cases.append({"case": name, "lam": lam, "batch": batch, "passes": passes})
            plan.close()
            del xs, out
            torch.cuda.empty_cache()
    print(json.dumps({"metric": "HBM GB/s of the FFT-form passes at lam <= 2", "unit": "GB/s", "peak": hbm,
                      "peak_source": f"hbm_gbs, {pk_src}", "form": "fold", "timing":
                      "CUDA events around each launch in a traced graph (event nodes add ~2-4 us per launch)",
                      "cases": cases}), flush=True)


# The companion record printed inside the line of a workload (the largest
# configuration has two lattices: the two-cloud 256^3 is the headline, the
# 128x128x1024 quasicondensate rides along as an extra record).
COMPANION = {"large_two_cloud": "large_quasicondensate"}
EXTRA_KEYS = ("value", "unit", "ms_per_step", "config", "rel_l2_density_err_vs_fp64", "gpu_launches",
              "clocks", "roofline", "roofline_hbm", "hbm_step", "pass_ms", "e2e")


def run_ffx(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1602_03395_gb300 import build as B
    B.build()
    from paper_1602_03395_gb300 import ffx

    if args.fft_passes:
        run_fft_passes(args, torch, dev, ffx)
        if world > 1:
            dist.destroy_process_group()
        return 0

    if args.workload == "mixed":
        rc = run_mixed(args, torch, dist, world, rank, dev)
        if world > 1:
            dist.destroy_process_group()
        return rc

    line = measure_workload(args, torch, dist, world, rank, local, dev, ffx, workload(args.workload, args.batch))
    extra = []
    if args.workload in COMPANION and not args.no_companion and args.column is None:
        torch.cuda.empty_cache()
        rec = measure_workload(args, torch, dist, world, rank, local, dev, ffx,
                               workload(COMPANION[args.workload], args.batch), primary=False)
        if rec is not None:
            extra.append({k: rec[k] for k in EXTRA_KEYS})
    if rank == 0:
        if extra:
            line["extra_records"] = extra
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ffx(args)


if __name__ == "__main__":
    sys.exit(main())
