"""Throughput benchmark of OCD soft-output detection on GB300.

Workload: 128 BS antennas x 8 users, 64-QAM, K = 3 sweeps, T = 14 OFDM
symbols per channel realization, 1200 data subcarriers per OFDM symbol
(2048-point OFDM), OCD-BOX at 15 dB.  One step detects FRAMES x 1200
subcarriers in one call (inputs ~540 MB, so every step streams from HBM and
no L2 flush is needed).  Metric: detected Gb/s = Nsc * T * U * Q bits / s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run: every rank detects its own batch
(subcarriers are independent; no data-path collective), the time is the
maximum over ranks and the value counts all ranks' bits (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

B, U, T, K, ORDER, Q = 128, 8, 14, 3, 64, 6
NSC_FRAME = 1200
FRAMES = 20
SNR_DB = 15.0
METRIC = "detected Gb/s (128x8, 64-QAM, K=3) and % HBM roofline vs plain FP32 form"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SMS_NOMINAL = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
# device sources of the headline kernel (its host launch code is not part of it)
KERNEL_SOURCES = ["ocd_common.cuh", "ocd_mma.cuh", "ocd_tma_util.cuh", "ocd_projected_tma.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ocd_projected_tma_128x8_t14_k3.md")
MIN_CLOCK_WINDOW_S = 0.5
REF_BUDGET_S = 60.0


def algorithmic_bytes_per_sc(b=B, u=U, t=T, q=Q):
    """H (8BU) + Y (8TB) read once, xhat (8TU) + LLR (4TUQ) written once."""
    return 8 * b * u + 8 * t * b + 8 * t * u + 4 * t * u * q


def algorithmic_bytes_per_sc_stored(b, u, t, q, elem):
    """As algorithmic_bytes_per_sc with H, Y stored at `elem` bytes per complex."""
    return elem * b * u + elem * t * b + 8 * t * u + 4 * t * u * q


def to16(x, dtype):
    """complex64 tensor -> contiguous [..., 2] tensor of a 16-bit dtype."""
    import torch
    return torch.view_as_real(x).to(dtype).contiguous()


def algorithmic_fma_per_sc(b=B, u=U, t=T, k=K):
    """Algorithm 1: 8BU real FMAs per (sweep, symbol) (Section III-B: one
    inner product and one scalar-by-vector product), plus 2BU for the norms."""
    return 8 * b * u * k * t + 2 * b * u


def kernel_source_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1611_08779_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    sha = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    val = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not sha or not val or sha.group(1) != kernel_source_sha():
        return None
    return float(val.group(1))


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, ValueError):
            self.proc = None
        # nvidia-smi's start-up (NVML initialization, first queries) competes
        # with the host side of the launches: the timed region starts only
        # after its first sample has arrived (at most 5 s)
        t0 = time.monotonic()
        while self.proc is not None and not self.lines and time.monotonic() - t0 < 5.0:
            if self.proc.poll() is not None:
                break
            time.sleep(0.02)
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=5)

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _oracle_sample(nsc_sample, seed):
    from paper_1611_08779_gb300 import synth
    return synth.make_uplink(nsc_sample, B, U, T, ORDER, SNR_DB, seed)


def cpu_oracle_rate(d, min_seconds, mode, impl="c", threads=0):
    """Time the FP64 oracle as it stands on the sample d (repeated until
    min_seconds have passed); returns (Gb/s, seconds, subcarriers processed).
    impl "c": the plain-C oracle, one subcarrier per OpenMP iteration over
    `threads` host threads (0: all); "numpy": the NumPy oracle (one thread)."""
    import oracle as orc
    m = orc.BOX if mode == "box" else orc.MMSE
    nsc = d["H"].shape[0]
    if impl == "c":
        from oracle import native
        native.build()

        def run():
            native.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, K, m, ORDER, threads=threads)
    else:
        def run():
            orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, K, m, ORDER)
    done, t0 = 0, time.perf_counter()
    while True:
        run()
        done += nsc
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return done * T * U * Q / el / 1e9, el, done


def oracle_threads():
    """Host threads of the C oracle's parallel loop (all cores unless
    OMP_NUM_THREADS says otherwise)."""
    from oracle import native
    return native.max_threads()


def cpu_baseline_line(args):
    """The C oracle on every host core over a bounded sample, with its
    single-core rate and the NumPy oracle's beside it."""
    d = _oracle_sample(NSC_FRAME, 99)
    r, el, done = cpu_oracle_rate(d, args.cpu_seconds, args.mode)
    d1 = {k: (v[: NSC_FRAME // 8] if k in ("H", "Y") else v) for k, v in d.items()}
    r1, el1, _ = cpu_oracle_rate(d1, args.cpu_seconds / 4, args.mode, threads=1)
    d2 = {k: (v[:24] if k in ("H", "Y") else v) for k, v in d.items()}
    r2, el2, _ = cpu_oracle_rate(d2, args.cpu_seconds / 4, args.mode, impl="numpy")
    return {
        "value": r, "unit": "Gb/s", "cores": oracle_threads(), "kind": "oracle",
        "sample": f"{NSC_FRAME} subcarriers x {T} symbols of the workload, {done // NSC_FRAME} "
                  f"times in {el:.1f} s (FP64 C oracle, all host cores)",
        "single_core_gbps": _r(r1), "numpy_oracle_gbps": _r(r2),
    }


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    nsc = args.frames * NSC_FRAME  # the workload of the other arm
    # Size each step's sample so the whole --steps/--warmup run stays near
    # REF_BUDGET_S seconds of oracle time (one calibration run first); one
    # sample of inputs is drawn once and detected every step.
    cal = _oracle_sample(NSC_FRAME // 4, 999)
    _, el, done = cpu_oracle_rate(cal, 0.0, args.mode)
    per_sc = el / done
    sample = int(REF_BUDGET_S / (per_sc * (args.steps + args.warmup)))
    sample = max(16, min(nsc, args.ref_sample, sample))
    d = _oracle_sample(sample, 1000)
    rates = []
    for i in range(args.warmup + args.steps):
        r, el, done = cpu_oracle_rate(d, 0.0, args.mode)
        if i >= args.warmup:
            rates.append((r, el))
    total_bits = len(rates) * sample * T * U * Q
    total_s = sum(el for _, el in rates)
    value = total_bits / total_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gb/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # one step of the workload at the measured rate; each timed step ran
        # a bounded sample of it (cpu_baseline.sample)
        "ms_per_step": 1e3 * nsc * T * U * Q / (value * 1e9),
        "sample_ms_per_step": 1e3 * total_s / len(rates), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, nsc),
        "cpu_baseline": {"value": value, "unit": "Gb/s", "cores": oracle_threads(),
                         "kind": "oracle",
                         "sample": f"{sample} of the {nsc} subcarriers x {T} symbols per step of "
                                   f"the 128x8 64-QAM K=3 workload, FP64 C oracle (one subcarrier "
                                   f"per OpenMP iteration, all host cores)"},
        "e2e": {"value": value, "unit": "Gb/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, nsc):
    return {"workload": f"OCD-{args.mode.upper()} 128x8 64-QAM K=3 T=14, "
                        f"{nsc} subcarriers per step per GPU",
            "B": B, "U": U, "T": T, "K": K, "qam": ORDER, "mode": args.mode,
            "snr_db": SNR_DB, "subcarriers_per_step": nsc,
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"subcarriers x{args.gpus}"}


def form_summary(measure, args):
    """One of the extra forms measured beside the headline number, reduced to
    its compact summary; a failure is reported in the object instead of
    losing the line."""
    import argparse as _ap
    sub = _ap.Namespace(**vars(args))
    sub.steps = min(args.steps, 50)
    try:
        res = measure(sub)
    except Exception as exc:  # reported, not hidden: the key says what failed
        return {"error": f"{type(exc).__name__}: {exc}"[:200]}
    return _r(res["summary"])


def _r(x, digits=4):
    """Floats of a summary rounded to `digits` significant digits (the line
    stays short enough to be kept whole by a log tail)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}") if math.isfinite(x) else x
    if isinstance(x, dict):
        return {k: _r(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_r(v, digits) for v in x]
    return x


SWEEP_SNR_DB = (0.0, 15.0, 30.0)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1611_08779_gb300 as ocd
    from paper_1611_08779_gb300 import synth

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    nsc = NSC_FRAME * args.frames
    d = synth.make_uplink(nsc, B, U, T, ORDER, SNR_DB, seed=7 + rank)
    H = torch.from_numpy(d["H"]).to(dev)
    Y = torch.from_numpy(d["Y"]).to(dev)
    xhat = torch.empty((nsc, T, U), dtype=torch.complex64, device=dev)
    llr = torch.empty((nsc, T, U, Q), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    N0 = d["N0"]
    peaks, src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    alg_bytes = algorithmic_bytes_per_sc() * nsc
    bits_per_step = nsc * T * U * Q * world

    def step():
        ocd.ocd_detect(H, Y, N0, 1.0, K, args.mode, ORDER, xhat=xhat, llr=llr, stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(ms):
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed_ms(fn, steps, warm=3):
        """Mean device time of one fn() on `stream` (CUDA events, warm-up
        untimed, synchronized on both sides), max over ranks."""
        with torch.cuda.stream(stream):
            for _ in range(warm):
                fn()
        barrier()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(steps):
                fn()
            ev1.record(stream)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1) / steps)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    barrier()
    sampler = ClockSampler(dev.index)
    with sampler:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1)
        # Short timed regions see too few clock samples: keep the same step
        # running (untimed) until the sampling window reaches half a second.
        hold = 0
        if ms < 1e3 * args.clock_window:
            hold = int((1e3 * args.clock_window - ms) / max(ms / args.steps, 1e-3)) + 1
            with torch.cuda.stream(stream):
                for _ in range(hold):
                    step()
            barrier()
    ms = max_over_ranks(ms)
    value = bits_per_step * args.steps / (ms / 1e3) / 1e9
    form_steps = max(3, min(args.steps, 50))

    # Both modes of Algorithm 1 over the SNR sweep of the metric configuration
    # (same channels, bits and noise draw; only the noise scale changes), the
    # same launch on the same stream.
    sweep = {}
    if not args.no_forms:
        for snr in SWEEP_SNR_DB:
            ds = synth.make_uplink(nsc, B, U, T, ORDER, snr, seed=7 + rank)
            Ys = torch.from_numpy(ds["Y"]).to(dev)
            del ds["H"], ds["Y"]
            for mode in ("box", "mmse"):
                msp = timed_ms(lambda: ocd.ocd_detect(H, Ys, ds["N0"], 1.0, K, mode, ORDER,
                                                      xhat=xhat, llr=llr, stream=stream),
                               form_steps)
                sweep.setdefault(mode, {})[f"{snr:g}"] = [
                    bits_per_step / world / (msp / 1e3) / 1e9,
                    alg_bytes / (msp / 1e3) / 1e9 / hbm_peak]
            del Ys
        barrier()

    # The residual arrangement (Algorithm 1 as written, r kept in full) on the
    # same inputs: the plain FP32 form the metric compares against.
    ms_res = timed_ms(lambda: ocd.ocd_detect(H, Y, N0, 1.0, K, args.mode, ORDER, xhat=xhat,
                                             llr=llr, stream=stream, algo="residual"),
                      form_steps)

    # Precision forms: the same batch with H and Y stored as bfloat16 / float16
    # pairs, timed the same way, and compared with the float32-storage outputs.
    forms = {}
    xr = xhat.clone()
    lr = llr.clone()
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        H16, Y16 = to16(H, dt), to16(Y, dt)
        x16 = torch.empty_like(xhat)
        l16 = torch.empty_like(llr)
        ms16 = timed_ms(lambda: ocd.ocd_detect(H16, Y16, N0, 1.0, K, args.mode, ORDER, xhat=x16,
                                               llr=l16, stream=stream),
                        max(3, min(args.steps, 200)))
        b16 = algorithmic_bytes_per_sc_stored(B, U, T, Q, 4) * nsc
        agree = float(((l16 > 0) == (lr > 0)).float().mean().item())
        forms[name] = {"gbps": bits_per_step / world / (ms16 / 1e3) / 1e9, "ms": ms16,
                       "hbm_frac": b16 / (ms16 / 1e3) / 1e9 / hbm_peak,
                       "bits_equal_f32": agree}
        del H16, Y16, x16, l16

    # End to end through the host-buffer entry point: pinned inputs copied in
    # and results copied out inside the timed region.  Its ceiling: the
    # pinned copies alone (one direction at a time, same bytes, same stream),
    # with the two directions and the kernel fully overlapped.
    Hh = torch.from_numpy(d["H"]).pin_memory()
    Yh = torch.from_numpy(d["Y"]).pin_memory()
    xh = torch.empty((nsc, T, U), dtype=torch.complex64, pin_memory=True)
    lh = torch.empty((nsc, T, U, Q), dtype=torch.float32, pin_memory=True)
    staging = {"H": H, "Y": Y, "X": xhat, "L": llr}
    h2d_bytes = int(Hh.numel() * 8 + Yh.numel() * 8)
    d2h_bytes = int(xh.numel() * 8 + lh.numel() * 4)

    def h2d():
        H.copy_(Hh, non_blocking=True)
        Y.copy_(Yh, non_blocking=True)

    def d2h():
        xh.copy_(xhat, non_blocking=True)
        lh.copy_(llr, non_blocking=True)

    ms_h2d = timed_ms(h2d, 3, warm=1)
    ms_d2h = timed_ms(d2h, 3, warm=1)

    def e2e_step():
        ocd.ocd_detect_host(Hh, Yh, N0, 1.0, K, args.mode, ORDER, xhat=xh, llr=lh,
                            staging=staging, pieces=args.pieces, device=dev, stream=stream)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    e2e_steps = max(1, min(args.steps, 5))
    ev0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    ev1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(ev0.elapsed_time(ev1))
    e2e_value = bits_per_step * e2e_steps / (ms_e2e / 1e3) / 1e9
    e2e_ceiling = bits_per_step / (max(ms_h2d, ms_d2h, ms / args.steps) / 1e3) / 1e9

    if rank == 0:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        per_launch_s = ms / 1e3 / args.steps
        achieved_gbs = alg_bytes / per_launch_s / 1e9
        traffic = recorded_traffic()
        clocks = sampler.summary()
        if clocks is not None:
            clocks["window"] = "timed region" if hold == 0 else \
                f"timed region + {hold} untimed identical steps"
        alu_peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
        res_tf = 2 * algorithmic_fma_per_sc() * nsc / (ms_res / 1e3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": "Gb/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (i.i.d. Rayleigh H, Gray 64-QAM, AWGN)",
            "config": workload_config(args, nsc),
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                         "peak_source": f"{src} hbm_gbs",
                         "kernel": "ocd_projected_tma_kernel",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "e2e": {"value": e2e_value, "unit": "Gb/s", "h2d_bytes_per_step": h2d_bytes,
                    "d2h_bytes_per_step": d2h_bytes, "pieces": args.pieces,
                    "h2d_gbs": h2d_bytes / (ms_h2d / 1e3) / 1e9,
                    "d2h_gbs": d2h_bytes / (ms_d2h / 1e3) / 1e9,
                    "ceiling_gbps": e2e_ceiling, "frac": e2e_value / e2e_ceiling},
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_line(args)
        # Forms measured beside the headline, last and rounded so that the
        # line stays short: [Gb/s, fraction of the HBM roofline] per point.
        line["snr_sweep"] = _r({"unit": "[Gb/s, hbm frac]", **sweep}) if sweep else None
        line["residual_form"] = _r({
            "gbps": bits_per_step / world / (ms_res / 1e3) / 1e9, "ms": ms_res,
            "alu_frac": res_tf / alu_peak, "kernel": "ocd_residual_kernel",
            "alu_peak_tflops": alu_peak})
        line["precision_forms"] = _r(forms)
        if not args.no_forms:
            line["batched_form"] = form_summary(measure_batched, args)
            line["unfolded_form"] = form_summary(measure_unfolded, args)
            line["single_symbol_form"] = form_summary(measure_single, args)
            line["wide_form"] = form_summary(measure_wide, args)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_precision(args):
    """256x16, 3300 subcarriers, T = 14, K = 4, 64-QAM with H and Y stored as
    float32, bfloat16 and float16 pairs: throughput of each (inputs 198 MB in
    float32 > L2), and per SNR the difference of the 16-bit forms from the
    float32-storage result and the uncoded bit error rate against the sent
    bits.  (The per-SNR error against the FP64 reference is measured by the
    test-suite: tests/test_precision_gpu.py.)"""
    import torch

    import paper_1611_08779_gb300 as ocd
    from paper_1611_08779_gb300 import synth
    b, u, t, k, q, nsc = 256, 16, 14, 4, 6, 3300
    dev = torch.device("cuda", 0)
    d = synth.make_uplink(nsc, b, u, t, ORDER, SNR_DB, seed=11)
    H = torch.from_numpy(d["H"]).to(dev)
    Y = torch.from_numpy(d["Y"]).to(dev)
    stores = {"f32": (H, Y, 8), "bf16": (to16(H, torch.bfloat16), to16(Y, torch.bfloat16), 4),
              "f16": (to16(H, torch.float16), to16(Y, torch.float16), 4)}
    peak = float(measured_peaks()[0].get("hbm_gbs", FALLBACK_HBM_GBS))
    out = {}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for name, (h, y, elem) in stores.items():
        x = torch.empty((nsc, t, u), dtype=torch.complex64, device=dev)
        llr = torch.empty((nsc, t, u, q), dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            ocd.ocd_detect(h, y, d["N0"], 1.0, k, args.mode, ORDER, xhat=x, llr=llr)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            ocd.ocd_detect(h, y, d["N0"], 1.0, k, args.mode, ORDER, xhat=x, llr=llr)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        nbytes = algorithmic_bytes_per_sc_stored(b, u, t, q, elem) * nsc
        out[name] = {"value": nsc * t * u * q / (ms / 1e3) / 1e9, "unit": "Gb/s",
                     "ms_per_step": ms, "hbm_frac": nbytes / (ms / 1e3) / 1e9 / peak}
    per_snr = {}
    for snr in range(0, 31, 5):
        ds = synth.make_uplink(480, b, u, t, ORDER, float(snr), seed=100 + snr)
        h32 = torch.from_numpy(ds["H"]).to(dev)
        y32 = torch.from_numpy(ds["Y"]).to(dev)
        x32, l32 = ocd.ocd_detect(h32, y32, ds["N0"], 1.0, k, args.mode, ORDER)
        x32 = x32.cpu().numpy()
        l32 = l32.cpu().numpy()
        row = {"f32": {"ber_vs_sent": float(np.mean((l32 > 0).astype(np.uint8) != ds["bits"]))}}
        for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
            x, l = ocd.ocd_detect(to16(h32, dt), to16(y32, dt), ds["N0"], 1.0, k, args.mode, ORDER)
            x = x.cpu().numpy()
            l = l.cpu().numpy()
            xe = np.max(np.linalg.norm(x - x32, axis=-1)
                        / np.maximum(np.linalg.norm(x32, axis=-1), 1e-3 * math.sqrt(u)))
            le = np.abs(l - l32) / np.maximum(np.abs(l32), 1.0)
            row[name] = {"xhat_rel_diff_vs_f32_max": float(xe),
                         "llr_rel_diff_vs_f32_p99": float(np.quantile(le, 0.99)),
                         "hard_bit_mismatch_vs_f32": float(np.mean((l > 0) != (l32 > 0))),
                         "ber_vs_sent": float(np.mean((l > 0).astype(np.uint8) != ds["bits"]))}
        per_snr[str(snr)] = row
    line = {"metric": "detected Gb/s, precision form (256x16, 64-QAM, K=4, T=14)",
            "workload": "precision", "unit": "Gb/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"OCD-{args.mode.upper()} 256x16 64-QAM K=4 T=14, "
                                   f"{nsc} subcarriers per step", "B": b, "U": u, "T": t, "K": k},
            "forms": out, "accuracy_per_snr_db": per_snr,
            "accuracy_sample": "480 subcarriers x 14 symbols per SNR; 16-bit forms against the "
                               "float32-storage result, and uncoded BER against the sent bits"}
    print(json.dumps(line), flush=True)
    return 0


SINGLE_CONFIGS = (  # (B, U, order, subcarriers per frame of --frames)
    (128, 8, 64, 4000),
    (32, 8, 16, 12000),
)


def measure_single(args):
    """One symbol per channel (T = 1, K = 3, OCD-BOX at 15 dB): 128x8 64-QAM
    and 32x8 16-QAM, whose inputs (frames x 4000 and frames x 12000
    subcarriers: 758 MB and 599 MB at 20 frames) stream from HBM; the
    one-lane-per-subcarrier projected kernel (what AUTO runs) against the
    HBM roofline, with the residual form beside it."""
    import torch

    import paper_1611_08779_gb300 as ocd
    from paper_1611_08779_gb300 import synth
    dev = torch.device("cuda", 0)
    peak = float(measured_peaks()[0].get("hbm_gbs", FALLBACK_HBM_GBS))
    stream = torch.cuda.Stream(dev)
    out = {}
    for b, u, order, per_frame in SINGLE_CONFIGS:
        q = int(round(math.log2(order)))
        nsc = per_frame * args.frames
        d = synth.make_uplink(nsc, b, u, 1, order, SNR_DB, seed=21)
        H = torch.from_numpy(d["H"]).to(dev)
        Y = torch.from_numpy(d["Y"]).to(dev)
        del d["H"], d["Y"]
        x = torch.empty((nsc, 1, u), dtype=torch.complex64, device=dev)
        llr = torch.empty((nsc, 1, u, q), dtype=torch.float32, device=dev)
        arms = {}
        for algo in ("auto", "residual"):
            def step():
                ocd.ocd_detect(H, Y, d["N0"], 1.0, K, args.mode, order, xhat=x, llr=llr,
                               algo=algo, stream=stream)
            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    step()
            torch.cuda.synchronize(dev)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            steps = args.steps if algo == "auto" else max(3, args.steps // 4)
            with torch.cuda.stream(stream):
                ev0.record(stream)
                for _ in range(steps):
                    step()
                ev1.record(stream)
            torch.cuda.synchronize(dev)
            arms[algo] = ev0.elapsed_time(ev1) / steps
        ms = arms["auto"]
        nbytes = algorithmic_bytes_per_sc(b, u, 1, q) * nsc
        achieved = nbytes / (ms / 1e3) / 1e9
        out[f"{b}x{u}"] = {
            "value": nsc * u * q / (ms / 1e3) / 1e9, "unit": "Gb/s", "ms_per_step": ms,
            "config": {"B": b, "U": u, "T": 1, "K": K, "qam": order, "mode": args.mode,
                       "subcarriers_per_step": nsc},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "kernel": "ocd_projected_lane_kernel",
                         "algorithmic_bytes_per_launch": nbytes},
            "residual_form": {"value": nsc * u * q / (arms["residual"] / 1e3) / 1e9,
                              "unit": "Gb/s", "ms_per_step": arms["residual"]},
        }
        del H, Y, x, llr
    summary = {"unit": "[Gb/s, hbm frac, residual-form Gb/s]", "kernel": "ocd_projected_lane_kernel"}
    for key, f in out.items():
        summary[key] = [f["value"], f["roofline"]["frac"], f["residual_form"]["value"]]
    return {"metric": "detected Gb/s, one symbol per channel (T=1, K=3)", "forms": out,
            "value": out["128x8"]["value"], "unit": "Gb/s",
            "ms_per_step": out["128x8"]["ms_per_step"], "summary": summary}


def run_single(args):
    res = measure_single(args)
    line = {"metric": res["metric"], "workload": "single", "value": res["value"], "unit": "Gb/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": "OCD-BOX T=1 K=3: 128x8 64-QAM and 32x8 16-QAM",
                       "l2": "inputs larger than L2 (no flush)"},
            "forms": res["forms"]}
    print(json.dumps(line), flush=True)
    return 0


WIDE_CONFIGS = (  # (B, U, T, K, order, subcarriers per step)
    (256, 32, 14, 4, 64, 4000),
    (128, 32, 14, 3, 64, 8000),
)


def measure_wide(args):
    """The projected form for 17-32 users (OCD-BOX at 15 dB): the
    tensor-memory (tcgen05) kernel against the warp-level MMA kernel on the
    same inputs (434 MB and 491 MB of algorithmic traffic per launch, inputs
    larger than L2), each against the HBM
    roofline of its algorithmic bytes."""
    import torch

    import paper_1611_08779_gb300 as ocd
    from paper_1611_08779_gb300 import synth
    dev = torch.device("cuda", 0)
    peak = float(measured_peaks()[0].get("hbm_gbs", FALLBACK_HBM_GBS))
    stream = torch.cuda.Stream(dev)
    out = {}
    for b, u, t, k, order, nsc in WIDE_CONFIGS:
        q = int(round(math.log2(order)))
        d = synth.make_uplink(nsc, b, u, t, order, SNR_DB, seed=23)
        H = torch.from_numpy(d["H"]).to(dev)
        Y = torch.from_numpy(d["Y"]).to(dev)
        del d["H"], d["Y"]
        x = torch.empty((nsc, t, u), dtype=torch.complex64, device=dev)
        llr = torch.empty((nsc, t, u, q), dtype=torch.float32, device=dev)
        nbytes = algorithmic_bytes_per_sc(b, u, t, q) * nsc
        row = []
        for algo in ("projected_tc", "projected_warp"):
            def step():
                ocd.ocd_detect(H, Y, d["N0"], 1.0, k, args.mode, order, xhat=x, llr=llr,
                               algo=algo, stream=stream)
            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    step()
            torch.cuda.synchronize(dev)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                ev0.record(stream)
                for _ in range(args.steps):
                    step()
                ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms = ev0.elapsed_time(ev1) / args.steps
            row += [nsc * t * u * q / (ms / 1e3) / 1e9, nbytes / (ms / 1e3) / 1e9 / peak, ms]
        out[f"{b}x{u}_t{t}_k{k}"] = row
        del H, Y, x, llr
    return {"metric": "detected Gb/s, 17-32 users", "forms": out,
            "summary": {"unit": "[tcgen05 Gb/s, hbm frac, ms, warp-level Gb/s, hbm frac, ms]",
                        **out}}


def run_wide(args):
    res = measure_wide(args)
    line = {"metric": res["metric"], "workload": "wide", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "OCD-BOX 256x32 T=14 K=4 and 128x32 T=14 K=3, 64-QAM",
                       "l2": "inputs larger than L2 (no flush)"},
            "forms": res["summary"]}
    print(json.dumps(line), flush=True)
    return 0


def batched_bound_s(spec, hbm_gbs, fma_tflops, projected):
    """Roofline time of one cell in the arrangement the batched form runs it
    in: the projected form is bound by HBM; the residual form by max(HBM,
    FP32 FMA: 8BU per sweep and symbol, Section III-B)."""
    b, u, t, k = spec["B"], spec["U"], spec["T"], spec["K"]
    q = int(round(math.log2(spec["order"])))
    nbytes = algorithmic_bytes_per_sc(b, u, t, q) * spec["Nsc"]
    t_hbm = nbytes / (hbm_gbs * 1e9)
    if projected:
        return t_hbm, nbytes
    t_alu = 2.0 * algorithmic_fma_per_sc(b, u, t, k) * spec["Nsc"] / (fma_tflops * 1e12)
    return max(t_hbm, t_alu), nbytes


def measure_batched(args):
    """Mixed cells in one call: (B, U) in {(32,4), (64,8), (128,16), (256,32)},
    T in {1, 7, 14}, Nsc uniform in [300, 3300], K in [2, 5], MMSE / BOX,
    16 / 64-QAM (seeded).  Arms: the plain form (one ocd_detect per cell on one
    stream), the batched persistent launch with default tiles, and the
    batched launch with autotuned tiles replayed as a CUDA graph; the default
    and tuned arms are timed alternately and their ratio reported."""
    import torch

    import paper_1611_08779_gb300 as ocd
    from paper_1611_08779_gb300 import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs = synth.mixed_cell_specs(args.cells, seed=12)
    cells, bits = [], 0
    for s in specs:
        d = synth.make_uplink(s["Nsc"], s["B"], s["U"], s["T"], s["order"], s["snr_db"], s["seed"])
        cells.append(ocd.make_cell(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["Y"]).to(dev),
                                   d["N0"], 1.0, s["K"], s["mode"], s["order"]))
        bits += s["Nsc"] * s["T"] * s["U"] * int(round(math.log2(s["order"])))
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fma_tf = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    ws = ocd.make_workspace(len(cells), dev)

    def per_cell():
        for c in cells:
            ocd.ocd_detect(c.H, c.Y, c.N0, c.Es, c.K, c.mode, c.qam_order, xhat=c.xhat, llr=c.llr)

    def timed(fn, steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    steps = max(3, min(args.steps, 200))
    arms = {}
    arms["per_cell_launches"] = timed(per_cell, steps)
    t0 = time.perf_counter()
    tune = ocd.ocd_autotune_batched(cells, reps=3, workspace=ws)
    tune_s = time.perf_counter() - t0
    algo_of = {(e["B"], e["U"], e["T"]): e["algo"] for e in tune.entries}
    projected = (2, 3, 4)  # OCD_ALGO_PROJECTED, _PROJECTED_WARP, _PROJECTED_TC
    bound = [batched_bound_s(s, hbm, fma_tf, algo_of[(s["B"], s["U"], s["T"])] in projected)
             for s in specs]
    t_bound = sum(b for b, _ in bound)
    nbytes = sum(n for _, n in bound)
    # default and tuned tiles timed alternately (three rounds, best of each),
    # so that a drift of the box between the two does not enter their ratio
    default_ms, tuned_ms = float("inf"), float("inf")
    for _ in range(3):
        default_ms = min(default_ms, timed(lambda: ocd.ocd_detect_batched(cells, workspace=ws),
                                           steps))
        tuned_ms = min(tuned_ms, timed(lambda: ocd.ocd_detect_batched(cells, tune=tune,
                                                                      workspace=ws), steps))
    arms["batched_default_tiles"] = default_ms
    arms["batched_tuned"] = tuned_ms
    graph = ocd.BatchedGraph(cells, tune=tune, workspace=ws)
    sampler = ClockSampler(dev.index)
    with sampler:
        arms["batched_tuned_graph"] = ms = timed(graph.launch, steps)
    graph.close()
    clocks = sampler.summary()
    value = bits / (ms / 1e3) / 1e9
    line = {
        "metric": "detected Gb/s, batched form (mixed cells in one persistent launch)",
        "workload": "batched", "value": value, "unit": "Gb/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic (i.i.d. Rayleigh H, Gray QAM, AWGN)",
        "config": {"workload": f"{len(cells)} mixed cells, {sum(s['Nsc'] for s in specs)} "
                               f"subcarriers, {bits} bits per step",
                   "cells": [{k: s[k] for k in ("B", "U", "T", "Nsc", "K", "mode", "order")}
                             for s in specs],
                   "l2": "inputs larger than L2 (no flush)"},
        "arms_gbps": {k: bits / (v / 1e3) / 1e9 for k, v in arms.items()},
        "arms_ms": arms,
        "roofline": {"bound": "mixed (hbm for cells the tuned plan runs in the projected form, "
                              "max(hbm, fp32) for residual-form cells)",
                     "bound_ms": t_bound * 1e3, "frac": t_bound * 1e3 / ms,
                     "hbm_achieved_gbs": nbytes / (ms / 1e3) / 1e9, "hbm_peak": hbm,
                     "fp32_peak_tflops": fma_tf, "peak_source": f"{src} hbm_gbs; FP32 nominal"},
        "tune": tune.entries, "tune_seconds": tune_s,
        "clocks": clocks,
    }
    short = {"per_cell_launches": "per_cell", "batched_default_tiles": "default",
             "batched_tuned": "tuned", "batched_tuned_graph": "tuned_graph"}
    line["tuned_over_default"] = default_ms / tuned_ms - 1.0
    line["summary"] = {"gbps": value, "ms": ms, "roofline_frac": t_bound * 1e3 / ms,
                       "arms_gbps": {short[k]: bits / (v / 1e3) / 1e9 for k, v in arms.items()},
                       "tuned_over_default": default_ms / tuned_ms - 1.0,
                       "cells": len(cells)}
    return line


def run_batched(args):
    print(json.dumps(measure_batched(args)), flush=True)
    return 0


def measure_unfolded(args):
    """Differentiable unfolded OCD-BOX: 128x16, K = 5, 4096 (subcarrier,
    symbol) samples (each its own channel), 16-QAM, SNR uniform in 5-25 dB per
    sample, BCE loss on the LLRs.  A step is forward + loss + adjoint."""
    import torch
    import torch.nn.functional as F

    import paper_1611_08779_gb300 as ocd
    from paper_1611_08779_gb300 import synth
    b, u, k, order, nsc = 128, 16, 5, 16, 4096
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(21)
    snr = rng.uniform(5.0, 25.0, size=nsc)
    n0 = 10.0 ** (-snr / 10.0)
    d = synth.make_uplink(nsc, b, u, 1, order, 100.0, seed=21)
    noise = rng.standard_normal(d["Y"].shape) + 1j * rng.standard_normal(d["Y"].shape)
    Y = (d["Y"] + noise * np.sqrt(n0 / 2.0)[:, None, None]).astype(np.complex64)
    H = torch.from_numpy(d["H"]).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    N0 = torch.from_numpy(n0.astype(np.float32)).to(dev)
    bits = torch.from_numpy(d["bits"].astype(np.float32)).to(dev)
    om = torch.full((k,), 0.9, device=dev, requires_grad=True)
    al = torch.full((k,), 0.05, device=dev, requires_grad=True)

    def step(arr="projected"):
        om.grad = None
        al.grad = None
        _, llr = ocd.unfolded_ocd(om, al, H, Yd, N0, 1.0, "box", order, algo=arr)
        loss = F.binary_cross_entropy_with_logits(llr, bits)
        loss.backward()
        return loss

    def step_fused():
        # the same loss formed where the forward kernel forms the LLRs
        om.grad = None
        al.grad = None
        loss = ocd.unfolded_bce_loss(om, al, H, Yd, N0, bits, 1.0, "box", order)
        loss.backward()
        return loss

    def fwd(arr="projected"):
        with torch.no_grad():
            ocd.unfolded_ocd(om, al, H, Yd, N0, 1.0, "box", order, algo=arr)

    def timed(fn, steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    steps = max(3, min(args.steps, 200))
    ms_fwd = timed(fwd, steps)
    ms_res = timed(lambda: step("residual"), steps)
    ms_eager = timed(step, steps)
    # The training step captured once in a CUDA graph (forward, loss,
    # adjoint and the gradient reduction), replayed: device time without the
    # host's per-step Python and launch overhead.  Timed: the fused loss
    # (forward kernel with the BCE and its LLR derivative, loss reduction,
    # adjoint, gradient reduction: four launches); beside it the composable
    # step (unfolded_ocd, then PyTorch's BCE and autograd kernels).
    def capture(fn):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            out = fn()
        return graph, out

    graph_c, _ = capture(step)
    ms_comp = timed(graph_c.replay, steps)
    graph, g_loss = capture(step_fused)
    sampler = ClockSampler(dev.index)
    with sampler:
        ms = timed(graph.replay, steps)
    q = 4
    samples = nsc
    # Algorithmic work of one step in the projected arrangement, per sample:
    # G (upper triangle) 2BU(U+1) and q0 4BU FMA, sweeps 4U per update in the
    # forward, the replay and the reverse (12KU^2); bytes: H and Y read once,
    # G and the (q, z) checkpoints written and read, xhat / LLR written and
    # read back, the LLR adjoint read.
    fma = samples * (2 * b * u * (u + 1) + 4 * b * u + 12 * k * u * u)
    nbytes = samples * (8 * b * u + 8 * b + 2 * 8 * u * u + 2 * k * 2 * u * 8
                        + 2 * (8 * u + 4 * u * q) + 4 * u * q)
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fma_tf = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    t_bound = max(nbytes / (hbm * 1e9), 2.0 * fma / (fma_tf * 1e12))
    line = {
        "metric": "training samples/s, unfolded OCD-BOX forward + adjoint (128x16, K=5, 16-QAM)",
        "workload": "unfolded", "value": samples / (ms / 1e3), "unit": "samples/s", "n_gpus": 1,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "forward_ms": ms_fwd,
        "arrangement": "projected (q = H^H r, G per sample)",
        "timing": "CUDA-graph replay of the whole step (forward with the fused BCE, loss "
                  "reduction, adjoint, gradient reduction)",
        "composable_ms_per_step": ms_comp,
        "eager_ms_per_step": ms_eager,
        "residual_arrangement_eager_ms_per_step": ms_res,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic (i.i.d. Rayleigh H, "
        "Gray 16-QAM, AWGN at SNR uniform 5-25 dB per sample)",
        "config": {"workload": f"{samples} samples of 128x16, K=5, T=1, BCE loss", "B": b, "U": u,
                   "K": k, "qam": order, "l2": "inputs 67 MB + checkpoints 13 MB (no flush)"},
        "roofline": {"bound": "max(hbm, fp32)", "bound_ms": t_bound * 1e3,
                     "frac": t_bound * 1e3 / ms, "achieved_tflops": 2.0 * fma / (ms / 1e3) / 1e12,
                     "achieved_gbs": nbytes / (ms / 1e3) / 1e9, "hbm_peak": hbm,
                     "fp32_peak_tflops": fma_tf, "peak_source": f"{src} hbm_gbs; FP32 nominal"},
        "loss": float(g_loss.detach()),
        "clocks": sampler.summary(),
    }
    line["summary"] = {"samples_per_s": samples / (ms / 1e3), "ms": ms, "forward_ms": ms_fwd,
                       "composable_ms": ms_comp, "roofline_frac": t_bound * 1e3 / ms}
    return line


def run_unfolded(args):
    print(json.dumps(measure_unfolded(args)), flush=True)
    return 0


def parser():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["box", "mmse"], default="box")
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--pieces", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-sample", type=int, default=NSC_FRAME * FRAMES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and unfolded forms in the headline line")
    ap.add_argument("--workload", choices=["metric", "precision", "batched", "unfolded", "single",
                                           "wide"],
                    default="metric",
                    help="metric: the headline 128x8 configuration; precision: 256x16 K=4 in "
                         "float32 / bfloat16 / float16 storage with per-SNR accuracy; batched: "
                         "mixed cells in one persistent launch; unfolded: differentiable OCD-BOX "
                         "forward + adjoint (128x16, K=5, 4096 samples); single: one symbol per "
                         "channel (T=1: 128x8 64-QAM, 32x8 16-QAM); wide: 17-32 users "
                         "(tcgen05 and warp-level kernels)")
    ap.add_argument("--cells", type=int, default=24, help="cells of the batched workload")
    ap.add_argument("--clock-window", type=float, default=MIN_CLOCK_WINDOW_S,
                    help="seconds of clock sampling the timed steps are extended to")
    return ap


def main(argv=None):
    ap = parser()
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "unfolded":
        return run_unfolded(args)
    if args.workload == "single":
        return run_single(args)
    if args.workload == "wide":
        return run_wide(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
