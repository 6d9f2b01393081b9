"""Throughput of the fused multichannel filter chain on GB300.

Workload (the configuration the headline metric is quoted on): 64 channels x
2,880,000 samples (60 s at 48 kHz) of seeded pink noise through an 8th-order
Chebyshev-I low-pass (4 sections), 4 peaking-EQ biquads and a 1025-tap
low-pass FIR (TorchFX, arXiv 2504.08624: Sec. 3 filter chain, Sec. 4
multichannel workloads).  One step = one pass of the whole chain over the
whole signal.  Inputs (737 MB) exceed the 129 MB L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "channel-samples/s through filter chain (fwd, fwd+bwd) vs plain GPU; % HBM roofline"
UNIT = "channel-samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--flags", type=int, default=0, help="TFX_PLAN_* bits for the timed plan")
    ap.add_argument("--channels", type=int, default=None, help="override channel count (testing only)")
    ap.add_argument("--samples", type=int, default=None, help="override samples per channel (testing only)")
    ap.add_argument("--clips", type=int, default=None, help="only the first K clips of the batched workload "
                                                             "(profiling only)")
    ap.add_argument("--workload", default="multichannel_fused",
                    choices=["multichannel_fused", "plain_chain", "long_fir", "table4_chain", "differentiable_chain",
                             "batched_clips", "paper_sweep"],
                    help="configuration to time (default: the one the headline metric is quoted on)")
    ap.add_argument("--part", choices=["chain", "iir", "fir"], default="chain",
                    help="time the whole chain (default) or only its IIR cascade / FIR stage (profiling)")
    ap.add_argument("--mode", choices=["fwd", "fwdbwd"], default=None,
                    help="step = forward pass (default), or training forward + MSE + backward "
                         "(default for the differentiable_chain workload)")
    ap.add_argument("--no-fwdbwd", action="store_true",
                    help="skip the fwd+bwd measurement added to a forward run")
    ap.add_argument("--no-long-fir", action="store_true",
                    help="skip the long-FIR precision measurement added to a forward run")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the many-clip batched measurement added to a forward run")
    args = ap.parse_args()
    if args.mode is None:
        args.mode = "fwdbwd" if args.workload == "differentiable_chain" else "fwd"
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args):
    from paper_2504_08624_gb300 import workloads as W
    if getattr(args, "workload", "") == "batched_clips":
        return None
    wl = W.WORKLOADS[getattr(args, "workload", "multichannel_fused")]()
    if args.channels:
        wl.C = args.channels
    if args.samples:
        wl.N = args.samples
    part = getattr(args, "part", "chain")
    if part == "iir":
        wl.stages = [st for st in wl.stages if st[0] == "sos"]
    elif part == "fir":
        wl.stages = [st for st in wl.stages if st[0] == "fir"]
    return wl


def algorithmic(wl):
    """Algorithmic work per channel-sample: 8 bytes (FP32 read + write, the
    signal crosses HBM once), 10 flop per SOS section, 2L flop per L-tap FIR."""
    S = sum(np.asarray(c).reshape(-1, 6).shape[0] for k, c in wl.stages if k == "sos")
    L = sum(np.asarray(c).size for k, c in wl.stages if k == "fir")
    return 8.0, 10.0 * S + 2.0 * L, S, L


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "source": "fallback"}


def n_units(stages) -> int:
    """Fused kernels one execution launches: consecutive SOS stages merge
    into one cascade and each FIR closes a unit (one launch per unit)."""
    n, pending = 0, False
    for kind, coef in stages:
        if kind == "sos":
            pending = pending or np.asarray(coef).size > 0
        else:
            n += 1
            pending = False
    return n + (1 if pending else 0)


def fp32_alu_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flop) per lane per clock (nominal, for context)
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_fp32_peak(dev, stream, torch, sm_count: int, local: int) -> dict:
    """The FP32 FMA rate of this GPU, measured: 8 CTAs of 256 threads per SM,
    each thread 8 independent FMA chains of 4096 steps (scalar, and the packed
    two-lane form), timed with CUDA events over 20 launches after 3 warm-ups,
    with the SM clock sampled meanwhile.  The CUDA-core rooflines divide by
    the larger of the two."""
    from paper_2504_08624_gb300 import _native as NAT
    lib = NAT.lib()
    blocks, threads, iters = sm_count * 8, 256, 4096
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    h = ctypes.c_void_p(stream.cuda_stream)
    res = {}
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    for packed in (0, 1):
        def run():
            NAT.check(lib.tfx_fma_probe(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters, packed, h),
                      "tfx_fma_probe")
        k = 20
        t = time_gpu(run, k, 3, stream, torch, None) / k
        res["fma2" if packed else "fma"] = lib.tfx_fma_probe_flops(blocks, threads, iters, packed) / t / 1e12
    clocks = sampler.stop()
    peak = max(res.values())
    return {"tflops": peak, "scalar_fma_tflops": res["fma"], "packed_fma2_tflops": res["fma2"], "clocks": clocks,
            "how": f"{blocks} CTAs x {threads} threads x 8 FMA chains x {iters} steps, best of scalar and "
                   "packed two-lane FMA, CUDA events over 20 launches"}


def channel_rel_err(got, ref, scale=None):
    """Per-channel max|got - ref| / max|ref| (or / scale when given)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1, np.asarray(got).shape[-1])
    ref = np.asarray(ref, dtype=np.float64).reshape(got.shape)
    err = np.max(np.abs(got - ref), axis=1)
    sc = np.max(np.abs(ref), axis=1) if scale is None else np.asarray(scale, dtype=np.float64)
    return err / np.maximum(sc, 1e-300)


def unit_stages(desc, stages):
    """Pair each unit of a plan description with the stages it runs: a
    cascade takes the SOS stages up to the next FIR, a fused unit those and
    the FIR, a FIR unit one FIR stage."""
    out, i = [], 0
    for u in desc:
        take = []
        if u["kind"] == "chain_fft":  # the whole chain in one unit
            out.append((u, list(stages)))
            i = len(stages)
            continue
        if u["kind"] in ("cascade", "fused"):
            while i < len(stages) and stages[i][0] == "sos":
                take.append(stages[i])
                i += 1
        if u["kind"] != "cascade" and i < len(stages) and stages[i][0] == "fir":
            take.append(stages[i])
            i += 1
        out.append((u, take))
    return out


def fft_flops_per_output(u) -> float:
    """Algorithmic flops per output of the FFT FIR: 5 M log2 M per complex
    transform of M points; single-block: a forward and an inverse transform
    and M complex products (6 flop) per two blocks of B outputs;
    partitioned: the two transforms and P complex multiply-adds (8 flop) per
    point per M outputs (two channels x B)."""
    M, B, P = u["M"], u["B"], u.get("P", 0)
    m = M.bit_length() - 1
    if P == 0:
        return (10.0 * M * m + 6.0 * M) / (2.0 * B)
    return (10.0 * M * m + 8.0 * P * M) / M


def kernel_name(u) -> str:
    """The kernel (or kernel pair) that runs one unit of a plan description."""
    k = u["kind"]
    if k == "fir_tc":
        return u["kernel"]
    if k == "fir_fft":
        return "k_fir_fft" if u.get("P", 0) == 0 else "k_fir_fft_spec+k_fir_fft_conv"
    if k == "chain_fft":
        return "k_fir_fft"
    if k == "cascade" and u.get("scan") == "tc":
        return "k_sos_tc"
    return {"warp": "k_sos_warp"}.get(u.get("scan"), "k_unit")


def unit_roofline(u, units, t, step_s, pk, fp32) -> dict:
    """One unit of a plan against its roofline (per-unit algorithmic work as
    stated in the module docstring).  The FFT FIR and the tensor-core cascade
    stream the signal once and do less arithmetic than direct filtering, so
    their bound is HBM at 8 B per sample; their own flop counts are stated
    beside it.  The tensor-core FIR is bound by the tensor pipe (2L flop per
    sample), the CUDA-core scans by the measured FP32 FMA rate (10 flop per
    section, 2L per fused FIR tap)."""
    k = u["kind"]
    row = {"route": k, "kernel_ms": t * 1e3, "share_of_step": t / step_s}
    hbm_ach = units * 8.0 / t / 1e9
    if k == "fir_tc":
        L = u["L"]
        K = -(-(L - 1) // 16) * 16 + 128
        row.update({"bound": "tensor", "kernel": u["kernel"], "achieved": units * 2.0 * L / t / 1e12,
                    "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                    "peak_source": f"{pk['source']} dense bf16/fp16 sustained",
                    "executed_tflops": units * 2.0 * 3 * K / t / 1e12,
                    "note": "achieved counts algorithmic 2L flop/sample; executed counts 3 split products x (W+128) K"})
    elif k in ("fir_fft", "chain_fft"):
        f = fft_flops_per_output(u)
        row.update({"bound": "hbm", "kernel": kernel_name(u), "achieved": hbm_ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "peak_source": f"{pk['source']} HBM copy bandwidth",
                    "config": {kk: u[kk] for kk in ("S", "L", "D", "Lc", "M", "B", "P") if kk in u},
                    "fft_tflops": units * f / t / 1e12,
                    "fft_frac_of_fp32": units * f / t / 1e12 / fp32["tflops"],
                    "note": f"8 B per sample (FP32 read + write); {f:.1f} transform flop per output "
                            "(5 M log2 M per transform) stated beside, against the measured FP32 FMA rate"})
    elif k == "cascade" and u.get("scan") == "tc":
        # tensor-core cascade: streams the signal once (8 B per sample); its tensor
        # work (GEMM1 128 x 112 and GEMM2 128 x 16 per 112-sample block, 3 split
        # products) takes under half the time the HBM traffic does at peak
        execf = 2.0 * 3 * 128 * (112 + 16) / 112
        row.update({"bound": "hbm", "kernel": kernel_name(u), "achieved": hbm_ach,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_source": f"{pk['source']} HBM copy bandwidth",
                    "executed_tflops": units * execf / t / 1e12,
                    "note": "8 B per sample (FP32 read + write); executed tensor flop per sample %.0f" % execf})
    else:
        S, L = u.get("S", 0), u.get("L", 0)
        row.update({"bound": "alu", "kernel": kernel_name(u),
                    "achieved": units * (10.0 * S + 2.0 * L) / t / 1e12, "peak": fp32["tflops"], "unit": "TFLOP/s",
                    "peak_source": "measured FP32 FMA rate (bench.measure_fp32_peak)",
                    "note": "10 flop per SOS section, 2L per FIR tap, per sample"})
        row["hbm_frac"] = hbm_ach / pk["hbm_gbs"]
    row["frac"] = row["achieved"] / row["peak"]
    return row


def measure_link(x_host, y_host, dev, torch, reps: int = 5) -> dict:
    """Copy-engine rate of the host link for these pinned buffers: host to
    device alone, device to host alone, and both at once on two streams
    (GB/s, CUDA events around each; the end-to-end step cannot beat the
    concurrent rate)."""
    d_in = torch.empty(x_host.shape, dtype=x_host.dtype, device=dev)
    d_out = torch.empty(y_host.shape, dtype=y_host.dtype, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    cur = torch.cuda.current_stream(dev)

    def run(fn):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(cur)
        for _ in range(reps):
            s1.wait_stream(cur)
            s2.wait_stream(cur)
            fn()
            cur.wait_stream(s1)
            cur.wait_stream(s2)
        b.record(cur)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    def h2d():
        with torch.cuda.stream(s1):
            d_in.copy_(x_host, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            y_host.copy_(d_out, non_blocking=True)

    def both():
        h2d()
        d2h()

    nb_in, nb_out = x_host.numel() * x_host.element_size(), y_host.numel() * y_host.element_size()
    t_in, t_out, t_both = run(h2d), run(d2h), run(both)
    del d_in, d_out
    return {"h2d": nb_in / t_in / 1e9, "d2h": nb_out / t_out / 1e9, "both": (nb_in + nb_out) / t_both / 1e9,
            "both_ms": t_both * 1e3}


def traffic_for(kernel: str, workload_name: str):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when the summary is missing or the kernel's sources (one file, or
    several hashed in order) changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel][workload_name]
        srcs = e["source"] if isinstance(e["source"], list) else [e["source"]]
        hs = hashlib.sha256()
        for src in srcs:
            hs.update(open(os.path.join(ROOT, src), "rb").read())
        h = hs.hexdigest()[:16]
        if h != e["source_sha256_16"]:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        self.out.close()
        os.unlink(self.out.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [v.strip() for v in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(t: float, dist, dev, torch) -> float:
    """The largest of every rank's value t (each rank receives it); t itself
    without a process group.  Timed regions report the slowest rank."""
    if dist is None:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def time_gpu(fn, steps, warmup, stream, torch, dist=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def cpu_oracle_rate(wl, C_sample: int, N_sample: int):
    """Time the FP64 oracle (as it stands) on a bounded sample; returns
    (channel-samples/s, seconds, threads)."""
    import oracle
    lib = oracle.load()
    x = wl.make_signal(C_sample, N_sample)
    t0 = time.perf_counter()
    lib.chain(x, wl.stages)
    dt = time.perf_counter() - t0
    return C_sample * N_sample / dt, dt, lib.num_threads()


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    if args.workload == "batched_clips":
        return reference_arm_batched(args)
    if args.workload == "paper_sweep":
        return reference_arm_sweep(args)
    wl = workload(args)
    ncpu = os.cpu_count() or 1
    Cs = min(wl.C, max(1, ncpu))
    Ns = min(wl.N, 240000)
    import oracle
    lib = oracle.load()
    x = wl.make_signal(Cs, Ns)
    for _ in range(args.warmup):
        lib.chain(x, wl.stages)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lib.chain(x, wl.stages)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    rate = Cs * Ns / dt
    sample = f"{Cs} channels x first {Ns} samples of the workload per step (FP64 oracle, OpenMP over channels)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "channels": wl.C, "samples": wl.N, "chain": chain_label(wl.stages)},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": lib.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def reference_arm_sweep(args):
    """The oracle on the paper's timing grid: each step filters a bounded
    sample (the first 240,000 samples of up to 12 channels) with each of the
    grid's two filters."""
    from paper_2504_08624_gb300 import workloads as W
    import oracle
    lib = oracle.load()
    Cs = min(max(W.PAPER_SWEEP_CHANNELS), max(1, os.cpu_count() or 1))
    Ns = 240000
    cells = [W.paper_sweep(k, max(W.PAPER_SWEEP_SECONDS), Cs) for k in ("fir", "iir")]
    xs = [wl.make_signal(Cs, Ns) for wl in cells]
    for _ in range(args.warmup):
        for wl, x in zip(cells, xs):
            lib.chain(x, wl.stages)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for wl, x in zip(cells, xs):
            lib.chain(x, wl.stages)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    rate = 2 * Cs * Ns / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "paper_sweep_44k1", "filters": {k: chain_label(wl.stages) for k, wl in
                                                              zip(("fir", "iir"), cells)}},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": lib.num_threads(), "kind": "oracle",
                         "sample": f"{Cs} channels x first {Ns} samples through each of the two filters per step "
                                   "(FP64 oracle, OpenMP over channels)"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


BWD_FLOP_PER_SECTION = 30.0  # recompute 10 + adjoint all-pole 4 + input gradient 6 + coefficient sums 10
FWDBWD_BYTES = 20.0          # fwd 8 (read x, write y) + bwd 12 (read g and x, write dx)
FWDBWD_BYTES_WITH_LOSS = 32.0  # plus the loss 12 (read y and the target, write g)


def fwdbwd_parity(wl, x, y, g, dx, torch, api, NAT) -> dict:
    """The timed training step's results against the FP64 oracle: the
    training forward's output on four whole channels, dL/dx at 56 sampled
    positions of the same channels (the oracle's impulse-response route,
    given the step's own dL/dy; scale: the channel's largest |dL/dx|), and the
    coefficient gradients of the same plan kind run on the first 8 channels
    (the oracle's vector-Jacobian product sums over exactly those)."""
    import oracle
    lib = oracle.load()
    chs = sorted({0, wl.C // 3, 2 * wl.C // 3, wl.C - 1})
    xs = x[chs].double().cpu().numpy()
    gs = g[chs].double().cpu().numpy()
    ys = y[chs].double().cpu().numpy()
    dxs = dx[chs].double().cpu().numpy()
    fwd_err = channel_rel_err(ys, lib.chain(xs, wl.stages))
    idx = np.unique(np.concatenate([np.linspace(0, wl.N - 1, 48).astype(np.int64),
                                    np.arange(max(0, wl.N - 8), wl.N)]))
    dx_err = []
    for i in range(len(chs)):
        ref = lib.chain_vjp_dx_at(gs[i], wl.stages, idx)
        dx_err.append(float(np.max(np.abs(dxs[i][idx] - ref)) / max(np.max(np.abs(dxs[i])), 1e-300)))
    Cs = min(8, wl.C)
    sub = api.Plan(Cs, wl.N, wl.stages, flags=NAT.TFX_PLAN_TRAINABLE)
    x8 = x[:Cs].contiguous()
    g8 = g[:Cs].contiguous()
    y8 = torch.empty_like(x8)
    dx8 = torch.empty_like(x8)
    dc8 = torch.empty(sub.coef_count, dtype=torch.float64, device=x.device)
    sv = sub.new_saved()
    sub.forward_train(x8, y8, sv)
    sub.backward(x8, g8, dx8, dc8, sv)
    torch.cuda.synchronize()
    if sub.get_error() != 0:
        raise RuntimeError("device reported a timeout in the parity backward")
    sub.close()
    _, grads = lib.chain_vjp(x8.double().cpu().numpy(), g8.double().cpu().numpy(), wl.stages, want_dx=False)
    got = dc8.cpu().numpy()
    coef_err, off = [], 0
    for (kind, _), gr in zip(wl.stages, grads):
        ref = gr.ravel()
        coef_err.append({"stage": kind, "max_rel_err": float(np.max(np.abs(got[off:off + ref.size] - ref)) /
                                                           max(np.max(np.abs(ref)), 1e-300))})
        off += ref.size
    return {"reference": "FP64 oracle", "tol_output": 1e-4, "tol_coef_grad": 1e-4,
            "forward_max_rel_err": float(fwd_err.max()), "forward_per_channel": [float(v) for v in fwd_err],
            "dx_max_rel_err": float(max(dx_err)), "dx_per_channel": dx_err, "channels": chs,
            "dx_positions": int(idx.size), "coef_grad": coef_err,
            "coef_grad_max_rel_err": float(max(e["max_rel_err"] for e in coef_err)),
            "coef_grad_channels": Cs,
            "note": "forward: whole channels; dL/dx: sampled positions, scale = the channel's largest |dL/dx|; "
                    "coefficient gradients: the first 8 channels through a plan of the same stages (per-stage "
                    "error relative to the stage's largest gradient)"}


def measure_fwdbwd(wl, steps, warmup, dev, stream, torch, dist, ws, rank, pk, sm_count, with_e2e, with_cpu,
                   fp32=None, with_parity=True):
    """One training step of the chain: training forward (saves chunk-start
    states), MSE against a target (loss and dL/dy in one kernel), backward
    (dL/dx and dL/d(every coefficient)).  Inputs resident in HBM."""
    from paper_2504_08624_gb300 import api, _native as NAT
    units = wl.C * wl.N
    S = sum(np.asarray(c).reshape(-1, 6).shape[0] for k, c in wl.stages if k == "sos")
    x_host = torch.from_numpy(wl.make_signal()).pin_memory()
    x = x_host.to(dev)
    # the target: the input through the same architecture with other parameters
    from paper_2504_08624_gb300 import workloads as W
    if "params" in wl.meta:
        tstages = W.differentiable_chain_target()
    else:
        tstages = [(k, (np.asarray(c) * np.array([1.1, 0.9, 1.05, 1, 1, 1]) if k == "sos"
                        else np.asarray(c) * 0.98)) for k, c in wl.stages]
    target = api.chain(x, tstages)
    plan = api.Plan(wl.C, wl.N, wl.stages, flags=NAT.TFX_PLAN_TRAINABLE)
    saved = plan.new_saved()
    fws = plan.workspace()
    bws = plan.backward_workspace()
    y = torch.empty_like(x)
    g = torch.empty_like(x)
    dx = torch.empty_like(x)
    dcoef = torch.empty(plan.coef_count, dtype=torch.float64, device=dev)

    lossbuf = torch.empty(1, dtype=torch.float64, device=dev)

    def fwd():
        plan.forward_train(x, y, saved, fws)

    def loss_step():
        return api.mse(y, target, g)

    def fwd_loss():  # the training forward with the loss fused (tfx_plan_forward_train_mse)
        plan.forward_train_mse(x, y, target, g, lossbuf, saved, fws)

    def bwd():
        plan.backward(x, g, dx, dcoef, saved, bws)

    tws = plan.train_workspace()

    def step():  # one call: forward, loss, backward (fused on the spectral route)
        plan.train_step_mse(x, y, target, g, lossbuf, dx, dcoef, saved, tws)

    def two_calls():  # the same step as forward_train_mse + backward
        fwd_loss()
        bwd()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t_eager = time_gpu(step, steps, 0, stream, torch, dist)
    # the same step captured once in a CUDA graph and replayed (no allocation
    # or host synchronisation inside the library calls, so they capture)
    graph = None
    try:
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        t = time_gpu(graph.replay, steps, warmup, stream, torch, dist)
    except Exception as exc:  # pragma: no cover - reported, eager timing kept
        graph = None
        t = t_eager
        graph_error = repr(exc)
    if plan.get_error() != 0:
        raise RuntimeError("device reported a timeout during the fwd+bwd run")
    t_all = max_over_ranks(t, dist, dev, torch)
    k_parts = max(5, steps // 4)
    t_f = time_gpu(fwd, k_parts, 2, stream, torch, None) / k_parts
    t_l = time_gpu(loss_step, k_parts, 2, stream, torch, None) / k_parts
    t_b = time_gpu(bwd, k_parts, 2, stream, torch, None) / k_parts
    t_fl = time_gpu(fwd_loss, k_parts, 2, stream, torch, None) / k_parts
    t_two = time_gpu(two_calls, k_parts, 2, stream, torch, None) / k_parts
    step()
    torch.cuda.synchronize()
    # y, g, dx and dcoef now hold one consistent training step
    parity = fwdbwd_parity(wl, x, y, g, dx, torch, api, NAT) if (with_parity and rank == 0) else None
    launches = plan.train_step_launches(True, True)
    step_s = t / steps

    route = plan.describe()
    roof = None
    parts = None
    if route and route[0]["kind"] == "chain_spectral":
        # spectral route: the step is one fused launch (forward, loss and the
        # correlation of g with x: read x and the target, write y and g,
        # 16 B per sample) with the coefficient gradients' four small
        # launches after it, and the input gradient (one reverse-time FFT
        # FIR: read g, write dx, 8 B per sample) on a side stream beside
        # them; each part timed alone through the plan's own calls
        k_k = max(10, steps // 3)
        t_dx = time_gpu(lambda: plan.backward(x, g, dx, None, saved, bws), k_k, 3, stream, torch, None) / k_k
        t_fz = time_gpu(lambda: plan.train_step_mse(x, y, target, g, lossbuf, None, dcoef, saved, tws), k_k, 3,
                        stream, torch, None) / k_k
        step()
        name_f = ("forward + MSE + correlation (k_fir_fft_train) + coefficient gradients (k_xcorr_reduce + "
                  "k_chain_grads_sec + k_chain_grads_fir + k_spectral_finalize)")
        parts = {name_f: t_fz, "dL/dx (k_fir_fft, reverse time)": t_dx}
        bytes_per = {name_f: 16.0, "dL/dx (k_fir_fft, reverse time)": 8.0}
        name, t_k = max(parts.items(), key=lambda kv: kv[1])
        ach = units * bytes_per[name] / t_k / 1e9
        kern = "k_fir_fft_train" if name == name_f else "k_fir_fft"
        roof = {"bound": "hbm", "kernel": kern, "part": name, "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "kernel_ms": t_k * 1e3, "share_of_step": t_k / step_s,
                "traffic": traffic_for(kern, wl.name), "peak_source": pk["source"],
                "route": route[0],
                "note": "algorithmic bytes per channel-sample of each part: the fused step 16 (read x and the "
                        "target, write y and g), dL/dx 8 (read g, write dx)"}
        parts = {k: v * 1e3 for k, v in parts.items()}
    elif S > 0:
        # dominant kernel: the cascade's reverse-time adjoint scan, timed alone
        # through a cascade-only trainable plan's backward with only dL/dx asked
        # (then that kernel is the only launch)
        sos_stages = [st for st in wl.stages if st[0] == "sos"]
        sp = api.Plan(wl.C, wl.N, sos_stages, flags=NAT.TFX_PLAN_TRAINABLE | NAT.TFX_PLAN_NO_COMPOSE)
        ssaved = sp.new_saved()
        sp.forward_train(x, y, ssaved)
        assert sp.backward_launches(True, False) == (S + 7) // 8
        k_k = max(10, steps // 3)
        t_k = time_gpu(lambda: sp.backward(x, g, dx, None, ssaved), k_k, 3, stream, torch, None) / k_k
        sp.close()
        alu_peak = fp32["tflops"] if fp32 else fp32_alu_peak_tflops(sm_count, pk["sm_max_mhz"])
        ach = units * BWD_FLOP_PER_SECTION * S / t_k / 1e12
        roof = {"bound": "alu", "kernel": "k_sos_bwd", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach / alu_peak, "kernel_ms": t_k * 1e3, "share_of_step": t_k / step_s,
                "traffic": traffic_for("k_sos_bwd", wl.name),
                "peak_source": "measured FP32 FMA rate (bench.measure_fp32_peak)" if fp32 else
                               f"{sm_count} SMs x 128 FP32 FMA x 2 flop x {pk['sm_max_mhz']:.0f} MHz (nominal)",
                "hbm_frac": units * 20.0 / t_k / 1e9 / pk["hbm_gbs"],
                "note": f"{BWD_FLOP_PER_SECTION:.0f} algorithmic flop per sample per section"}
    ach_gbs = units * FWDBWD_BYTES / step_s / 1e9
    hbm = {"bound": "hbm", "achieved": ach_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": ach_gbs / pk["hbm_gbs"], "peak_source": pk["source"],
           "frac_with_loss_bytes": units * FWDBWD_BYTES_WITH_LOSS / step_s / 1e9 / pk["hbm_gbs"],
           "note": f"{FWDBWD_BYTES:.0f} B per channel-sample: forward 8 (read x, write y), backward 12 "
                   f"(read g and x, write dx); with the MSE loss's 12 B it is {FWDBWD_BYTES_WITH_LOSS:.0f}"}

    e2e = None
    if with_e2e:
        # the public API a training loop calls: host batch and target copied in,
        # the FilterChain module forward, the fused MSE loss, autograd backward,
        # the loss and coefficient gradients read back
        t_host = target.cpu().pin_memory()
        if "params" in wl.meta:
            pr = wl.meta["params"]
            model = api.LearnableBiquadChain(pr["rho"], pr["phi"], pr["b"], pr["h"]).to(dev)
        else:
            model = api.FilterChain(wl.stages).to(dev)
        opt = torch.optim.SGD(model.parameters(), lr=1e-3)

        def e2e_step():
            opt.zero_grad(set_to_none=True)
            xd = x_host.to(dev, non_blocking=True)
            td = t_host.to(dev, non_blocking=True)
            loss = api.mse_loss(model(xd), td)
            loss.backward()
            opt.step()
            return float(loss.detach())

        w_e, k_e = 3, max(5, min(steps // 5, 30))
        t_e = time_gpu(e2e_step, k_e, w_e, stream, torch, dist)
        t_e = max_over_ranks(t_e, dist, dev, torch)
        e2e = {"value": units * ws * k_e / t_e, "unit": UNIT, "h2d_bytes_per_step": int(2 * units * 4),
               "d2h_bytes_per_step": int(8 + 8 * plan.coef_count), "ms_per_step": t_e / k_e * 1e3, "steps": k_e,
               "api": f"{type(model).__name__} (parameters on the GPU) + mse_loss + loss.backward() + SGD step; "
                      "the plan's coefficients updated on the device each step"}

    cpu = None
    if with_cpu and rank == 0 and ws == 1:
        import oracle
        lib = oracle.load()
        # a few seconds on the host cores: the oracle's dL/dx is O(N^2) per channel
        Cs = min(wl.C, 16)
        Ns = min(wl.N, 16384)
        xs = wl.make_signal(Cs, Ns).astype(np.float64)
        gs = np.random.default_rng(5).standard_normal(xs.shape)
        t0 = time.perf_counter()
        lib.chain(xs, wl.stages)
        lib.chain_vjp(xs, gs, wl.stages)
        dt = time.perf_counter() - t0
        cpu = {"value": Cs * Ns / dt, "unit": UNIT, "cores": lib.num_threads(), "kind": "oracle",
               "sample": f"{Cs} channels x first {Ns} samples: FP64 oracle chain + vector-Jacobian product "
                         f"(dL/dx from the impulse response, O(N^2) per channel; coefficient sensitivities), "
                         f"{dt:.1f} s"}
    plan.close()
    return {"workload": wl.name, "value": units * ws * steps / t_all, "unit": UNIT, "ms_per_step": step_s * 1e3,
            "steps": steps, "step": "one training step through tfx_plan_train_step_mse: forward, MSE loss and "
                                    "dL/dy, backward (dL/dx, dL/dcoef); on the spectral route the forward, the "
                                    "loss and the coefficient gradients' correlation are one launch",
            "two_calls_ms": t_two * 1e3,
            "cuda_graph": graph is not None, "eager_ms_per_step": t_eager / steps * 1e3,
            "fwd_ms": t_f * 1e3, "loss_ms": t_l * 1e3, "fwd_loss_ms": t_fl * 1e3, "bwd_ms": t_b * 1e3,
            "gpu_launches_per_step": launches,
            "route": route, "parts_ms": parts,
            "roofline": roof, "roofline_hbm": hbm, "e2e": e2e, "cpu_baseline": cpu, "parity": parity,
            "dtype": "f32", "plain_gpu": None}


def reference_arm_batched(args):
    """The oracle on the first clips of the many-clip workload (a bounded sample per step)."""
    import oracle
    from paper_2504_08624_gb300 import workloads as W
    lib = oracle.load()
    clips = W.batched_clips()[:8]
    xs = [c.make_signal() for c in clips]
    n = sum(c.C * c.N for c in clips)
    for _ in range(args.warmup):
        for c, x in zip(clips, xs):
            lib.chain(x, c.stages)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for c, x in zip(clips, xs):
            lib.chain(x, c.stages)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    rate = n / dt
    sample = f"first {len(clips)} clips ({n} channel-samples) per step, FP64 oracle, OpenMP over channels"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched_clips_1000"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": lib.num_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


LONG_FIR_ROUTES = [("fft", 0), ("tensor cores, FP16 hi/lo split", "TFX_PLAN_FIR_TC"),
                   ("tensor cores, BF16 hi/lo split", "TFX_PLAN_FIR_BF16_SPLIT"),
                   ("tensor cores, plain BF16 (reported only)", "TFX_PLAN_FIR_BF16_PLAIN")]


def measure_long_fir_precision(dev, stream, torch) -> dict:
    """The long-FIR configuration (128 x 4,194,304 Gaussian noise, 16384-tap
    Kaiser band-pass) on a bounded channel sample: its first 16 channels at
    full length through each FIR route, the error of each against the FP64
    oracle at 8 channels x 544 sampled outputs (the oracle's convolution at
    chosen positions; 32 of them within the first 16384 samples, where fewer
    than L terms enter), relative to the channel's largest |y| (from the
    default route's whole output), and each route's time beside."""
    from paper_2504_08624_gb300 import api, _native as NAT, workloads as W
    import oracle
    wl = W.WORKLOADS["long_fir"]()
    C = 16
    h = np.asarray(wl.stages[0][1], dtype=np.float64)
    xh = wl.make_signal(C, wl.N)
    x = torch.from_numpy(xh).to(dev)
    y = torch.empty_like(x)
    chs = list(range(0, C, 2))
    idx = np.unique(np.concatenate([np.linspace(0, wl.N - 1, 512).astype(np.int64),
                                    np.linspace(0, h.size - 1, 32).astype(np.int64)]))
    lib = oracle.load()
    ref = np.stack([lib.fir_at(xh[c].astype(np.float64), h, idx) for c in chs])
    out, scale = [], None
    for name, flag in LONG_FIR_ROUTES:
        flags = getattr(NAT, flag) if flag else 0
        plan = api.Plan(C, wl.N, wl.stages, flags=flags)
        wsb = plan.workspace()
        k = 5
        t = time_gpu(lambda: plan.execute(x, y, wsb), k, 2, stream, torch, None) / k
        torch.cuda.synchronize()
        if plan.get_error() != 0:
            raise RuntimeError(f"device reported a timeout on the long FIR ({name})")
        desc = plan.describe()
        plan.close()
        yc = y[chs]
        if scale is None:
            scale = yc.abs().amax(dim=1).double().cpu().numpy()
        got = yc[:, torch.from_numpy(idx).to(dev)].double().cpu().numpy()
        rel = channel_rel_err(got, ref, scale)
        out.append({"route": name, "plan": desc, "ms": t * 1e3, "channel_samples_per_s": C * wl.N / t,
                    "max_rel_err": float(rel.max()), "per_channel": [float(v) for v in rel],
                    "meets_1e-5": bool(rel.max() <= 1e-5)})
    return {"workload": f"{wl.name} (first {C} of {wl.C} channels, full length)", "taps": int(h.size),
            "reference": "FP64 oracle at sampled outputs", "tol": 1e-5, "channels_checked": chs,
            "positions_per_channel": int(idx.size), "routes": out}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return

    import torch
    from paper_2504_08624_gb300 import api, _native as NAT

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    dev = torch.device("cuda", local)
    if args.workload == "batched_clips":
        run_batched_main(args, dev, torch, dist, ws, rank, local)
        return
    if args.workload == "paper_sweep":
        run_paper_sweep_main(args, dev, torch, dist, ws, rank, local)
        return
    wl = workload(args)
    bytes_ps, flops_ps, S, L = algorithmic(wl)
    units = wl.C * wl.N

    if args.mode == "fwdbwd":
        run_fwdbwd_main(args, wl, dev, torch, dist, ws, rank, local)
        return

    x_host = torch.from_numpy(wl.make_signal()).pin_memory()
    x = x_host.to(dev)
    y = torch.empty_like(x)
    x_fir = torch.empty_like(x)
    plan = api.Plan(wl.C, wl.N, wl.stages, flags=args.flags)
    wsb = plan.workspace()
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.execute(x, y, wsb)

    # device-resident throughput (the headline `value`)
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_dev = time_gpu(step, args.steps, 0, stream, torch, dist)
    clocks = sampler.stop()
    err = plan.get_error()
    if err != 0:
        raise RuntimeError(f"device reported {NAT.STATUS.get(err, err)} during the timed run")
    t_all = max_over_ranks(t_dev, dist, dev, torch)
    value = units * ws * args.steps / t_all
    ms = t_all / args.steps * 1e3

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        y_host = torch.empty_like(x_host).pin_memory()

        def e2e_step():
            api.chain(x_host, wl.stages, out=y_host)

        w_e2e, k_e2e = max(3, min(args.warmup, 5)), max(5, min(args.steps // 10, 30))
        t_e2e = time_gpu(e2e_step, k_e2e, w_e2e, stream, torch, dist)
        t_e2e = max_over_ranks(t_e2e, dist, dev, torch)
        e2e = {"value": units * ws * k_e2e / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(x_host.numel() * 4), "d2h_bytes_per_step": int(y_host.numel() * 4),
               "ms_per_step": t_e2e / k_e2e * 1e3, "steps": k_e2e}
        # the host link's own bound: the same bytes copied in and out at once
        # by the copy engines (two streams, pinned buffers), no filtering
        link = measure_link(x_host, y_host, dev, torch)
        step_s = t_e2e / k_e2e
        e2e["link"] = {"gbs_concurrent": link["both"], "gbs_h2d": link["h2d"], "gbs_d2h": link["d2h"],
                       "copy_only_ms": link["both_ms"],
                       "frac": (x_host.numel() + y_host.numel()) * 4 / step_s / 1e9 / link["both"],
                       "note": "end-to-end bytes per step / step time, against the measured concurrent "
                               "host->device + device->host copy rate of the same buffers"}

    # the same chain with its units kept separate (no composite response), for context
    separate = None
    if any(u["kind"] == "chain_fft" for u in plan.describe()):
        splan = api.Plan(wl.C, wl.N, wl.stages, flags=args.flags | NAT.TFX_PLAN_NO_COMPOSE)
        sws = splan.workspace()
        k_s = max(10, args.steps // 5)
        t_s = time_gpu(lambda: splan.execute(x, x_fir, sws), k_s, 3, stream, torch, None) / k_s
        separate = {"ms_per_step": t_s * 1e3, "value": units / t_s, "plan": splan.describe(),
                    "launches": splan.launches_per_execute}
        splan.close()
        del sws

    # the plain sequential-per-channel GPU path on the same GB300
    plain = None
    if not args.no_plain:
        def plain_step():
            plan.execute(x, y, wsb, plain=True)
        k_plain = 2
        t_plain = time_gpu(plain_step, k_plain, 1, stream, torch, dist)
        plain = {"value": units * k_plain / t_plain, "unit": UNIT, "ms_per_step": t_plain / k_plain * 1e3,
                 "speedup": (units * args.steps / t_dev) / (units * k_plain / t_plain)}

    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    fp32 = measure_fp32_peak(dev, stream, torch, sm_count, local)
    step_s = t_dev / args.steps
    achieved_gbs = units * bytes_ps / step_s / 1e9
    # every unit of the chain timed alone (a plan of the unit's stages, same
    # flags, so the same kernels and launch configuration as inside the
    # chain, CUDA events on the launch stream); the dominant one against its
    # roofline
    unit_rows = []
    for u, ust in unit_stages(plan.describe(), wl.stages):
        uplan = api.Plan(wl.C, wl.N, ust, flags=args.flags)
        uws = uplan.workspace()
        k_u = max(10, args.steps // 3)
        t_u = time_gpu(lambda: uplan.execute(x, x_fir, uws), k_u, 3, stream, torch, None) / k_u
        uplan.close()
        del uws
        row = unit_roofline(u, units, t_u, step_s, pk, fp32)
        row["traffic"] = traffic_for(row["kernel"], wl.name)
        unit_rows.append(row)
    bound = max(unit_rows, key=lambda r: r["kernel_ms"]) if unit_rows else {
        "bound": "hbm", "kernel": "copy", "achieved": achieved_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    bound = dict(bound)
    bound["frac"] = bound["achieved"] / bound["peak"]
    bound["traffic"] = traffic_for(bound["kernel"], wl.name)
    hbm = {"bound": "hbm", "achieved": achieved_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": achieved_gbs / pk["hbm_gbs"], "peak_source": pk["source"],
           "note": "8 B per channel-sample over the whole step"}

    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        lib = oracle.load()
        ncpu = os.cpu_count() or 1
        Cs = min(wl.C, ncpu)
        # bounded sample: about 1.6e11 multiply-adds (10-30 s on the host cores)
        macs = max(1.0, flops_ps / 2.0)
        Ns = int(min(wl.N, max(16384, 1.6e11 / (Cs * macs))))
        xs = x_host[:Cs, :Ns].double().numpy()
        t0 = time.perf_counter()
        ref = lib.chain(xs, wl.stages)
        dt = time.perf_counter() - t0
        thr = lib.num_threads()
        cpu = {"value": Cs * Ns / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{Cs} of {wl.C} channels x first {Ns} of {wl.N} samples, FP64 oracle chain, "
                         f"{dt:.1f} s on {thr} threads"}
        # the same oracle on one thread (about 3e9 multiply-adds of the first channel)
        N1 = int(min(Ns, max(16384, 3e9 / macs)))
        lib.set_num_threads(1)
        t0 = time.perf_counter()
        lib.chain(xs[:1, :N1], wl.stages)
        dt1 = time.perf_counter() - t0
        lib.set_num_threads(thr)
        cpu["single_core"] = {"value": N1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"channel 0 x first {N1} samples, {dt1:.1f} s on 1 thread"}
        # the timed plan's output on the same channels (causal: the first Ns
        # outputs depend on the first Ns inputs only) against the oracle's
        step()
        torch.cuda.synchronize()
        got = y[:Cs, :Ns].double().cpu().numpy()
        rel = channel_rel_err(got, ref)
        parity = {"reference": "FP64 oracle", "tol": wl.tol, "max_rel_err": float(rel.max()),
                  "per_channel": [float(v) for v in rel], "channels": Cs, "samples": Ns,
                  "pass": bool(rel.max() <= wl.tol),
                  "note": "per channel: max|y - y_oracle| / max|y_oracle| over the channel, the timed plan's output"}

    fwd_bwd = None
    if not args.no_fwdbwd and args.part == "chain":
        from paper_2504_08624_gb300 import workloads as W
        fwd_bwd = measure_fwdbwd(W.differentiable_chain_forward(), min(args.steps, 100), max(3, args.warmup), dev,
                                 stream, torch, dist, ws, rank, pk, sm_count, not args.no_e2e,
                                 rank == 0 and ws == 1 and not args.no_cpu_baseline, fp32,
                                 with_parity=not args.no_cpu_baseline)
    long_fir = None
    if not args.no_long_fir and args.part == "chain" and rank == 0:
        long_fir = measure_long_fir_precision(dev, stream, torch)
    batched = None
    if not args.no_batched and args.part == "chain":
        batched = measure_batched(dev, stream, torch, dist, ws, rank, local, pk, fp32, 10, 3,
                                  with_e2e=not args.no_e2e, with_plain=False, with_cpu=False,
                                  with_parity=not args.no_cpu_baseline)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name if args.part == "chain" else f"{wl.name} ({args.part} only)",
                       "channels": wl.C, "samples": wl.N,
                       "chain": f"{S} SOS sections + FIR of {L} taps",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "inputs 737 MB > 129 MB L2, no flush", "plan_flags": args.flags},
            "roofline": bound, "roofline_hbm": hbm, "units": unit_rows, "cpu_baseline": cpu, "e2e": e2e,
            "parity": parity, "plain_gpu": plain, "separate_units": separate, "plan": plan.describe(),
            "gpu_launches": int(args.steps * plan.launches_per_execute),
            "clocks": clocks, "gpu": props.name, "fp32_peak": fp32, "fwd_bwd": fwd_bwd,
            "long_fir_precision": long_fir, "batched": batched,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def measure_batched(dev, stream, torch, dist, ws, rank, local, pk, fp32, steps, warmup, with_e2e=True,
                    with_plain=True, with_cpu=True, with_parity=True, nclips=None) -> dict:
    """The many-clip workload: 1000 clips, each its own length, channel count
    and chain, filtered by the batched launches (composed chains by FFT, one
    launch per transform size; the other clips' units grouped by level and
    kernel) replayed from one CUDA graph, with the autotuned parameters."""
    from paper_2504_08624_gb300 import api, autotune, workloads as W
    clips = W.batched_clips()
    if nclips:
        clips = clips[:nclips]
    spec = [(c.C, c.N, c.stages) for c in clips]
    total = sum(C * Ns for C, Ns, _ in spec)
    gen = torch.Generator(device=dev).manual_seed(5)
    x = torch.rand(total, device=dev, generator=gen) * 2 - 1
    cands = [{"fir_nb": nb, "tc_min_taps": t} for nb in (128, 256) for t in (64, 128)]
    t0 = time.perf_counter()
    tuned = autotune.tune_batch(spec, reps=2, candidates=cands)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = api.Batch(spec, fir_nb=tuned["fir_nb"], tc_min_taps=tuned["tc_min_taps"], fft_m=tuned["fft_m"])
    plan_s = time.perf_counter() - t0
    y = b.empty()
    wsb = b.workspace()
    parity = None
    if with_parity and rank == 0:
        # a sample of clips with their seeded signals against the oracle
        import oracle
        sample = [i for i in (0, 17, 333, 998) if i < len(clips)]
        xp = x.clone()
        for i in sample:
            b.view(xp, i).copy_(torch.from_numpy(clips[i].make_signal()))
        yp = b.execute(xp)
        torch.cuda.synchronize()
        errs = []
        for i in sample:
            c = clips[i]
            n = min(c.N, 200000)
            xs = np.ascontiguousarray(c.make_signal()[:, :n])
            got = b.view(yp, i).cpu().numpy().astype(np.float64)[:, :n]
            errs.append(float(channel_rel_err(got, oracle.chain(xs, c.stages)).max()))
        parity = {"reference": "FP64 oracle", "clips": sample, "max_rel_err": max(errs), "per_clip": errs,
                  "tol": 1e-4, "note": "first 200000 samples of each sampled clip, per channel"}
        del xp, yp
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        b.execute(x, y, wsb)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.execute(x, y, wsb)
    sampler = ClockSampler(local)
    for _ in range(max(3, warmup)):
        graph.replay()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t = time_gpu(graph.replay, steps, 0, stream, torch, dist)
    clocks = sampler.stop()
    if b.get_error() != 0:
        raise RuntimeError("device reported a timeout during the batched run")
    t_all = max_over_ranks(t, dist, dev, torch)
    step_s = t / steps
    # every launch timed alone; the dominant one against its roofline
    groups = []
    for g, (kind, level, tiles, samples, flops) in enumerate(b.groups()):
        k_g = 5
        t_g = time_gpu(lambda: b.execute_group(g, x, y, wsb), k_g, 2, stream, torch, None) / k_g
        groups.append({"kind": ["fused cascade+FIR", "cascade", "tensor-core FIR", "composed chain (FFT)",
                                "FFT FIR"][kind],
                       "level": level,
                       "tiles": tiles, "channel_samples": samples, "ms": t_g * 1e3,
                       "algorithmic_tflops": flops / t_g / 1e12})
    dom = max(range(len(groups)), key=lambda i: groups[i]["ms"])
    dg = groups[dom]
    if dg["kind"] == "tensor-core FIR":
        roof = {"bound": "tensor", "kernel": "k_fir_tc_batched", "peak": pk["bf16_tflops_sustained"],
                "peak_source": f"{pk['source']} dense bf16/fp16 sustained", "achieved": dg["algorithmic_tflops"],
                "unit": "TFLOP/s"}
    elif dg["kind"] in ("composed chain (FFT)", "FFT FIR"):
        roof = {"bound": "hbm", "kernel": "k_fir_fft_batched", "peak": pk["hbm_gbs"],
                "peak_source": f"{pk['source']} HBM copy bandwidth", "unit": "GB/s",
                "achieved": dg["channel_samples"] * 8.0 / (dg["ms"] * 1e-3) / 1e9,
                "note": "8 B per sample (FP32 read + write) of the group's clips"}
    else:
        roof = {"bound": "alu", "kernel": "k_unit_batched", "peak": fp32["tflops"],
                "peak_source": "measured FP32 FMA rate (bench.measure_fp32_peak)", "achieved": dg["algorithmic_tflops"],
                "unit": "TFLOP/s"}
    roof.update({"kernel_ms": dg["ms"], "share_of_step": dg["ms"] / (step_s * 1e3),
                 "traffic": traffic_for(roof["kernel"], "batched_clips")})
    roof["frac"] = roof["achieved"] / roof["peak"]
    ach_gbs = total * 8.0 / step_s / 1e9
    hbm = {"bound": "hbm", "achieved": ach_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": ach_gbs / pk["hbm_gbs"], "peak_source": pk["source"], "note": "8 B per channel-sample"}
    e2e = None
    if with_e2e:
        x_host = x.cpu().pin_memory()
        y_host = torch.empty_like(x_host).pin_memory()
        xd = torch.empty_like(x)

        def e2e_step():
            xd.copy_(x_host, non_blocking=True)
            b.execute(xd, y, wsb)
            y_host.copy_(y, non_blocking=True)

        k_e = 3
        t_e = time_gpu(e2e_step, k_e, 1, stream, torch, dist)
        e2e = {"value": total * ws * k_e / t_e, "unit": UNIT, "h2d_bytes_per_step": int(total * 4),
               "d2h_bytes_per_step": int(total * 4), "ms_per_step": t_e / k_e * 1e3, "steps": k_e,
               "api": "packed pinned host buffers, Batch.execute"}
        del x_host, y_host, xd
    plain = None
    if with_plain:
        # the plain sequential path on the first 20 clips (it runs at ~1e8 ch-samples/s)
        ps = [api.Plan(C, Ns, st) for C, Ns, st in spec[:20] if C * Ns > 0]
        xs = [torch.rand(p.C, p.N, device=dev) for p in ps]
        ys = [torch.empty_like(v) for v in xs]
        n_pl = sum(p.C * p.N for p in ps)
        t_p = time_gpu(lambda: [p.execute(a, o, plain=True) for p, a, o in zip(ps, xs, ys)], 1, 1, stream, torch,
                       None)
        plain = {"value": n_pl / t_p, "unit": UNIT, "sample": f"first {len(ps)} clips ({n_pl} channel-samples)",
                 "speedup": (total / step_s) / (n_pl / t_p)}
        for p in ps:
            p.close()
    cpu = None
    if with_cpu and rank == 0 and ws == 1:
        import oracle
        lib = oracle.load()
        t0 = time.perf_counter()
        n_cpu = 0
        for c in clips:
            if time.perf_counter() - t0 > 15.0:
                break
            xs_c = c.make_signal()
            lib.chain(xs_c, c.stages)
            n_cpu += c.C * c.N
        dt = time.perf_counter() - t0
        cpu = {"value": n_cpu / dt, "unit": UNIT, "cores": lib.num_threads(), "kind": "oracle",
               "sample": f"clips in order until 15 s ({n_cpu} channel-samples incl. signal generation), {dt:.1f} s"}
    out = {
        "workload": f"batched_clips_{len(clips)}", "value": total * ws * steps / t_all, "unit": UNIT,
        "ms_per_step": step_s * 1e3, "steps": steps,
        "config": {"workload": f"batched_clips_{len(clips)}", "clips": len(clips), "channel_samples": total,
                   "chains": "1-8 random stable sections + 33-2049-tap FIR per clip",
                   "launches": b.launches_per_execute, "cuda_graph": True,
                   "autotuned": {k: tuned[k] for k in ("fir_nb", "tc_min_taps", "fft_m", "cached")},
                   "tune_s": tune_s, "plan_s": plan_s,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": f"{total * 4 / 1e9:.1f} GB in and out per step > 129 MB L2, no flush"},
        "roofline": roof, "roofline_hbm": hbm, "groups": groups, "cpu_baseline": cpu, "e2e": e2e,
        "plain_gpu": plain, "parity": parity, "gpu_launches": int(steps * b.launches_per_execute),
        "clocks": clocks,
    }
    b.close()
    del x, y, wsb
    torch.cuda.empty_cache()
    return out


def run_batched_main(args, dev, torch, dist, ws, rank, local):
    """--workload batched_clips: the many-clip batch is the timed step."""
    stream = torch.cuda.current_stream(dev)
    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    fp32 = measure_fp32_peak(dev, stream, torch, props.multi_processor_count, local)
    r = measure_batched(dev, stream, torch, dist, ws, rank, local, pk, fp32, min(args.steps, 30), args.warmup,
                        not args.no_e2e, not args.no_plain, not args.no_cpu_baseline, not args.no_cpu_baseline,
                        nclips=args.clips)
    if rank == 0:
        out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": r["steps"],
               "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": r["config"]}
        out.update({k: r[k] for k in ("roofline", "roofline_hbm", "groups", "cpu_baseline", "e2e", "plain_gpu",
                                      "parity", "gpu_launches", "clocks")})
        out["gpu"] = props.name
        out["fp32_peak"] = fp32
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def chain_label(stages) -> str:
    """Short description of a chain's stages, in order."""
    parts = []
    for k, c in stages:
        if k == "sos":
            parts.append(f"{np.asarray(c).reshape(-1, 6).shape[0]} SOS")
        else:
            parts.append(f"FIR {np.asarray(c).size}")
    return " + ".join(parts)


def measure_paper_sweep(dev, stream, torch, dist, pk, reps, warmup, with_cpu):
    """The paper's timing grid (Sec. 4, Tables 2 and 3): each filter (a
    101-tap FIR and a 4th-order Butterworth, separately) on every cell of
    durations x channels of 44.1 kHz Gaussian noise; per cell the median of
    `reps` calls, each timed by its own pair of CUDA events (the paper's
    protocol: the median of 50 calls after warm-up), the plan built
    untimed.  The cells read prefixes of one resident 12 x 600 s buffer (row
    stride = the full length) and write into a second one."""
    from paper_2504_08624_gb300 import api, workloads as W
    secs, chans = W.PAPER_SWEEP_SECONDS, W.PAPER_SWEEP_CHANNELS
    top = W.paper_sweep("fir", max(secs), max(chans))
    Cmax, Nmax = top.C, top.N
    x = torch.from_numpy(top.make_signal()).to(dev)
    y = torch.empty_like(x)
    cells, launches = [], 0
    for kind in ("fir", "iir"):
        for sec in secs:
            for C in chans:
                wl = W.paper_sweep(kind, sec, C)
                plan = api.Plan(C, wl.N, wl.stages, ld=Nmax)
                wsb = plan.workspace()
                xv, yv = x[:C, :wl.N], y[:C, :wl.N]
                for _ in range(warmup):
                    plan.execute(xv, yv, wsb)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps)]
                torch.cuda.synchronize()
                if dist is not None:
                    dist.barrier()
                for a, b in ev:
                    a.record(stream)
                    plan.execute(xv, yv, wsb)
                    b.record(stream)
                torch.cuda.synchronize()
                err = plan.get_error()
                if err != 0:
                    raise RuntimeError(f"{wl.name}: plan status {err}")
                ts = [a.elapsed_time(b) / 1e3 for a, b in ev]
                med = max_over_ranks(statistics.median(ts), dist, dev, torch)
                mean = max_over_ranks(statistics.fmean(ts), dist, dev, torch)
                launches += reps * plan.launches_per_execute
                desc = plan.describe()
                cells.append({"filter": kind, "seconds": sec, "channels": C, "samples": wl.N,
                              "median_s": med, "mean_s": mean, "value": C * wl.N / med,
                              "hbm_frac": 8.0 * C * wl.N / med / (pk["hbm_gbs"] * 1e9),
                              "route": [u["kind"] for u in desc], "kernel": "+".join(kernel_name(u) for u in desc),
                              "M": [u.get("M") for u in desc]})
                plan.close()
    total_cs = sum(c["channels"] * c["samples"] for c in cells)
    total_t = sum(c["median_s"] for c in cells)
    # the dominant kernel: the filter whose cells take the larger share of
    # the grid's time, at its largest cell (one kernel per cell)
    share = {k: sum(c["median_s"] for c in cells if c["filter"] == k) for k in ("fir", "iir")}
    kd = max(share, key=share.get)
    big = max((c for c in cells if c["filter"] == kd), key=lambda c: c["channels"] * c["samples"])
    achieved = 8.0 * big["channels"] * big["samples"] / big["median_s"] / 1e9
    roof = {"bound": "hbm", "kernel": big["kernel"], "cell": f"{kd} {big['seconds']} s x {big['channels']} ch",
            "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
            "share_of_step": share[kd] / total_t, "traffic": None, "peak_source": pk["source"],
            "note": "8 algorithmic bytes per channel-sample (FP32 read + write); the cell's median call time"}
    cpu, parity = None, None
    if with_cpu:
        # the oracle on the 60 s x 12 channel cell of each filter: timed as it
        # stands (the CPU baseline) and compared with that cell's GPU output
        import oracle
        lib = oracle.load()
        n_cpu, t_cpu, parity = 0, 0.0, {"reference": "FP64 oracle", "cells": []}
        for kind in ("fir", "iir"):
            wl = W.paper_sweep(kind, 60, max(chans))
            plan = api.Plan(wl.C, wl.N, wl.stages, ld=Nmax)
            plan.execute(x[:wl.C, :wl.N], y[:wl.C, :wl.N], plan.workspace())
            got = y[:wl.C, :wl.N].cpu().numpy()
            plan.close()
            xs = wl.make_signal()
            t0 = time.perf_counter()
            ref = lib.chain(xs, wl.stages)
            t_cpu += time.perf_counter() - t0
            n_cpu += wl.C * wl.N
            e = channel_rel_err(got, ref)
            parity["cells"].append({"filter": kind, "seconds": 60, "channels": wl.C, "tol": wl.tol,
                                    "max_rel_err": float(max(e)), "per_channel": [float(v) for v in e]})
        parity["max_rel_err"] = max(c["max_rel_err"] for c in parity["cells"])
        cpu = {"value": n_cpu / t_cpu, "unit": UNIT, "cores": lib.num_threads(), "kind": "oracle",
               "sample": f"the 60 s x {max(chans)} channel cell of each filter ({n_cpu} channel-samples), "
                         f"FP64 oracle, {t_cpu:.1f} s"}
    return {"value": total_cs / total_t, "ms_per_step": total_t * 1e3, "cells": cells, "roofline": roof,
            "cpu_baseline": cpu, "parity": parity, "gpu_launches": launches,
            "filters": {k: chain_label(W.paper_sweep(k, 5, 1).stages) for k in ("fir", "iir")},
            "grid": {"seconds": list(secs), "channels": list(chans), "fs": W.PAPER_SWEEP_FS}}


def run_paper_sweep_main(args, dev, torch, dist, ws, rank, local):
    """--workload paper_sweep: the paper's timing grid; a step is one pass
    over all of its cells (value = all cells' channel-samples / the sum of
    their median call times)."""
    stream = torch.cuda.current_stream(dev)
    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    reps = max(1, min(args.steps, 50))
    r = measure_paper_sweep(dev, stream, torch, dist, pk, reps, max(3, args.warmup), not args.no_cpu_baseline)
    clocks = sampler.stop()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": r["value"] * ws, "unit": UNIT, "n_gpus": ws, "steps": reps,
            "warmup": max(3, args.warmup), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper_sweep_44k1", "grid": r["grid"], "filters": r["filters"],
                       "timing": "per cell: median (and mean) of the per-call CUDA-event times",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "no flush, as the paper's repeated calls: cells whose input and output fit in the "
                             "129 MB L2 stay resident between calls"},
            "roofline": r["roofline"], "cells": r["cells"], "cpu_baseline": r["cpu_baseline"],
            "parity": r["parity"], "e2e": None, "gpu_launches": r["gpu_launches"], "clocks": clocks,
            "gpu": props.name,
        }), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_fwdbwd_main(args, wl, dev, torch, dist, ws, rank, local):
    """--mode fwdbwd: the training step is the timed step (headline value)."""
    stream = torch.cuda.current_stream(dev)
    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    fp32 = measure_fp32_peak(dev, stream, torch, props.multi_processor_count, local)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    r = measure_fwdbwd(wl, args.steps, args.warmup, dev, stream, torch, dist, ws, rank, pk,
                       props.multi_processor_count, not args.no_e2e, not args.no_cpu_baseline, fp32,
                       with_parity=not args.no_cpu_baseline)
    clocks = sampler.stop()
    if rank == 0:
        S = sum(np.asarray(c).reshape(-1, 6).shape[0] for k, c in wl.stages if k == "sos")
        L = sum(np.asarray(c).size for k, c in wl.stages if k == "fir")
        print(json.dumps({
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "mode": "fwd+bwd", "channels": wl.C, "samples": wl.N,
                       "chain": f"{S} SOS sections + FIR of {L} taps, MSE loss",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": f"signals {wl.C * wl.N * 4 / 1e6:.0f} MB each, several per step > 129 MB L2, no flush"},
            "roofline": r["roofline"], "roofline_hbm": r["roofline_hbm"], "cpu_baseline": r["cpu_baseline"],
            "e2e": r["e2e"], "plain_gpu": r["plain_gpu"],
            "gpu_launches": int(args.steps * r["gpu_launches_per_step"]), "clocks": clocks, "gpu": props.name,
            "fwd_ms": r["fwd_ms"], "loss_ms": r["loss_ms"], "fwd_loss_ms": r["fwd_loss_ms"], "bwd_ms": r["bwd_ms"],
            "two_calls_ms": r["two_calls_ms"], "parts_ms": r["parts_ms"], "parity": r["parity"],
            "fp32_peak": fp32,
        }), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
