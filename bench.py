#!/usr/bin/env python3
"""Benchmark of the GB300 FZ-GPU compression path.

A step is one pass of the whole path over one field: fz_compress (value-
range-relative bound: range pass + fused compression kernel) followed by
fz_decompress, through the C ABI.  The workload is the 512^3 float32
lognormal Gaussian-random-field (spectrum k^-11/3) at relative bound 1e-3
(the stand-in for the paper's Nyx 512^3 field, Table 1), resident in HBM
before timing.  The field (512 MiB) is larger than L2 (129 MB), so
iterations need no L2 flush.

Printed (rank 0, one JSON line): round-trip GB/s of fp32 input (both
directions, 2 * 4N bytes per step over the device-timed step), compress and
decompress GB/s with p50/p99 latency, the dominant kernel's roofline
fraction against the measured HBM copy bandwidth, the end-to-end figure
through the host-buffer C-ABI calls, and the CPU oracle timed on a bounded
sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own field (independent problems: weak
scaling, no collective on the data path).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("compress+decompress GB/s of fp32 input (round trip, rel eb 1e-3); "
          "compress/decompress GB/s and p50/p99 latency alongside")
WORKLOAD = "cosmo3d_512"
WORKLOAD_DESC = ("512x512x512 float32 lognormal density exp(0.5 g), g a unit-std "
                 "Gaussian random field with power spectrum k^-11/3 (seed 3); "
                 "value-range-relative error bound 1e-3")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each kernel on the 512^3 workload: the mean of two warmed-up launches of one
# ncu capture of that kernel alone (-k, -c 2) in this benchmark.  A figure
# stands only while the kernel's sources are the ones that were captured
# (SHA-256 over them); otherwise the line reports null.
TRAFFIC = {
    "compress_kernel": (("fz_compress.cu", "fz_compress_impl.cuh", "fz_device.cuh", "fz_kernels.h"),
                        "8c61d73e4d3195fee77cbc77f0ba7a511e9fb5cabd2d0cd008f1ba8f3e5100f7",
                        537672576 + 74919040),
    "decompress_kernel": (("fz_decompress.cu", "fz_device.cuh", "fz_kernels.h"),
                          "9a4ecdaf0440f24d52cabaabb509476f96cc22b35f1f1b46b07fea78ea169ea3",
                          96723968 + 473442176),
    "range_kernel": (("fz_compress.cu", "fz_device.cuh", "fz_kernels.h"),
                     "81f361a7b3e5df991fa82e4717e8f1385841517c67bdc4a50a971338d86473b5",
                     536896256 + 1744768),
}


def traffic_bytes(kernel: str, size: int):
    """Captured DRAM bytes per launch, or None (other size, changed sources)."""
    import hashlib
    if size != 512 or kernel not in TRAFFIC:
        return None
    files, digest, nbytes = TRAFFIC[kernel]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2304_12557_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return nbytes if h.hexdigest() == digest else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo, hi = int(k), min(int(k) + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"fz_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9])
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_field(slab=None, size=512):
    from paper_2304_12557_gb300 import fields
    x = fields.cosmo3d(size)
    if slab is not None:
        x = x[:slab].copy()
    return x


def cpu_oracle_round_trip(x, reps=1, all_cores=False):
    """Time the CPU oracle (as it stands: one thread, or its all-cores
    variant) compress+decompress."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(reps):
        st, s = oracle.compress(x, 3, oracle.EB_REL, 1e-3, all_cores=all_cores)
        assert st == oracle.OK
        st, _ = oracle.decompress(s, all_cores=all_cores)
        assert st == oracle.OK
    return time.perf_counter() - t0, len(s)


def run_cpu_baseline_table(args, rank):
    """The cpu_baseline leg over the configurations: the CPU oracle as it
    stands timed on the host cores, compress and decompress separately, on the
    64^3 bumps, the 1800x3600 climate-like and the 512^3 lognormal fields at
    relative bounds 1e-2, 1e-3 and 1e-4: once single-threaded and once with
    the all-cores variant, whose streams and reconstructions must equal the
    single-threaded ones byte for byte (rank 0 only; no GPU work)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2304_12557_gb300 import fields
    oracle.build()
    cfgs = [("bumps3d_64", fields.bumps3d(64), 3), ("climate2d_1800x3600", fields.climate2d(), 2),
            ("cosmo3d_512", fields.cosmo3d(512), 3)]
    rows = []
    for name, x, ndim in cfgs:
        nbytes = 4 * x.size
        for eb in (1e-2, 1e-3, 1e-4):
            row = {"field": name, "rel_eb": eb}
            ref = None
            for label, all_cores in (("one_thread", False), ("all_cores", True)):
                t0 = time.perf_counter()
                st, s = oracle.compress(x, ndim, oracle.EB_REL, eb, all_cores=all_cores)
                t1 = time.perf_counter()
                assert st == oracle.OK, (name, eb, st)
                st, y = oracle.decompress(s, x.size, all_cores=all_cores)
                t2 = time.perf_counter()
                assert st == oracle.OK, (name, eb, st)
                if ref is None:
                    ref = (s, y.tobytes())
                    row["ratio"] = nbytes / len(s)
                else:
                    row["all_cores_identical"] = s == ref[0] and y.tobytes() == ref[1]
                row[label] = {"compress_gbs": nbytes / (t1 - t0) / 1e9,
                              "decompress_gbs": nbytes / (t2 - t1) / 1e9,
                              "compress_s": t1 - t0, "decompress_s": t2 - t1}
            rows.append(row)
    print(json.dumps({"metric": "CPU oracle compress/decompress GB/s of fp32 input per field and bound",
                      "value": None, "unit": "GB/s",
                      "config": {"workload": "cpu_baseline",
                                 "fields": [c[0] for c in cfgs], "rel_eb": [1e-2, 1e-3, 1e-4]},
                      "cpu_baseline": {"kind": "oracle", "cores": oracle.threads(),
                                       "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                                       "sample": "each field whole, one compress and one "
                                                 "decompress per variant and bound"},
                      "rows": rows}), flush=True)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_reference(args, rank):
    """The reference arm: the CPU oracle timed on the host cores on a bounded
    slab of the same workload per step (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    slab = 32
    x = make_field(slab)
    n = x.size
    for _ in range(args.warmup):
        cpu_oracle_round_trip(x, all_cores=True)
    times = []
    for _ in range(args.steps):
        t, _ = cpu_oracle_round_trip(x, all_cores=True)
        times.append(t)
    ms = 1e3 * sum(times) / len(times)
    value = 2 * 4 * n / (ms / 1e3) / 1e9
    cores = oracle.threads()
    sample = (f"512x512x{slab} slab of the 512^3 field, compress+decompress per step, "
              f"the oracle's all-cores variant on {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores,
                         "kind": "oracle", "sample": sample, "cpu_model": cpu_model(),
                         "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank, dist):
    import numpy as np
    import torch

    import paper_2304_12557_gb300 as fz
    from paper_2304_12557_gb300 import build

    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    x_h = make_field(size=args.size)
    n = x_h.size
    S = args.size
    field_bytes = 4 * n
    x_d = torch.from_numpy(x_h).to(dev)
    codec = fz.Codec(local_rank)
    stream = torch.cuda.current_stream(dev)
    cap = fz.stream_min_bytes((S, S, S), 3) + 16 * 256 * (n // 2048 + 64)
    s_d = torch.empty(cap, dtype=torch.uint8, device=dev)
    y_d = torch.empty_like(x_d)

    # One step: the whole fz_compress call, then the whole fz_decompress
    # call, each bracketed by CUDA events on the stream (so a call's time
    # includes its launches, its result read-back and its synchronisation).
    def step(rec):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        st, size = codec.compress_into(x_d, s_d, "rel", 1e-3, 3)
        e1.record(stream)
        codec.decompress_into(s_d, y_d, nbytes=size)
        e2.record(stream)
        if rec is not None:
            rec.append((e0, e1, e2, size))
        return size

    for _ in range(max(args.warmup, 3)):
        size = step(None)
    torch.cuda.synchronize()
    # correctness gate on the timed configuration (stream header sanity and
    # the pointwise bound on a sample); full parity lives in the tests
    info = fz.inspect(s_d[:64].cpu().numpy().tobytes())
    idx = torch.randint(0, n, (1 << 20,), device=dev, generator=torch.Generator(dev).manual_seed(1))
    err = (x_d.view(-1)[idx] - y_d.view(-1)[idx]).abs().max().item()
    assert err <= info["eb"] * (1 + 1e-5) + 2 ** -22 * float(x_d.abs().max()), err

    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ
                           else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank]))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    # the sampler runs through 0.3 s of untimed steps right before the timed
    # region and through the region itself, so that its samples see the GPU
    # under this load
    sampler.start()
    t_load = time.time()
    while time.time() - t_load < 0.3:
        step(None)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    recs = []
    t_start.record(stream)
    for _ in range(args.steps):
        step(recs)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    comp_ms = [a.elapsed_time(b) for a, b, _, _ in recs]
    dec_ms = [b.elapsed_time(c) for _, b, c, _ in recs]
    size = recs[-1][3]

    # A second timed pass with the library's whole-call events (recorded on
    # the stream at each call's entry and after its result read-back): each
    # fz_compress / fz_decompress call's own time, without the binding's.
    codec.set_call_timing(True)
    call_c, call_d = [], []
    for _ in range(args.steps):
        codec.compress_into(x_d, s_d, "rel", 1e-3, 3)
        codec.decompress_into(s_d, y_d, nbytes=size)
        cc, cd = codec.call_times_ms()
        call_c.append(cc)
        call_d.append(cd)
    codec.set_call_timing(False)

    # A third timed pass with the library's per-kernel CUDA events (recorded
    # on the launching stream around every kernel): each kernel's duration,
    # for the kernel-level roofline.
    codec.set_profiling(True)
    kc_all, kd_all = [], []
    for _ in range(args.steps):
        codec.compress_into(x_d, s_d, "rel", 1e-3, 3)
        kc_all.append(codec.kernel_times_ms())
        codec.decompress_into(s_d, y_d, nbytes=size)
        kd_all.append(codec.kernel_times_ms())
    codec.set_profiling(False)
    k_range = [kc[0] for kc in kc_all]
    k_comp = [kc[1] for kc in kc_all]
    k_out = [kc[2] for kc in kc_all]
    k_dec = [kd[3] for kd in kd_all]
    k_doff = [kd[4] for kd in kd_all]
    # per step: range, compress, (outliers), offsets pass, decompress
    launches = args.steps * (4 + (1 if max(k_out) > 0 else 0))

    mean = lambda v: sum(v) / len(v)
    peak, peak_kind = peaks()
    kern = {
        "compress_kernel": (mean(k_comp), field_bytes + size),
        "decompress_kernel": (mean(k_dec), size + field_bytes),
        "range_kernel": (mean(k_range), field_bytes),
    }
    dom = max(kern, key=lambda k: kern[k][0])
    achieved = kern[dom][1] / (kern[dom][0] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_bytes(dom, args.size),
            "peak_source": f"{peak_kind} hbm_gbs",
            "algorithmic_bytes_per_launch": kern[dom][1],
            "traffic_unit": "bytes per launch (ncu DRAM read + write)",
            "kernels": {k: {"ms": v[0], "GB/s": v[1] / (v[0] / 1e3) / 1e9,
                            "frac": v[1] / (v[0] / 1e3) / 1e9 / peak,
                            "traffic": traffic_bytes(k, args.size)}
                        for k, v in kern.items()}}
    # The two directions as kernel sequences: relative-bound compression is
    # the range pass plus the compressor, whose algorithmic bytes are two
    # reads of the input and the stream (8 + 4/CR bytes per element);
    # decompression is the offsets pass plus the decompressor (4/CR + 4).
    rel_ms = mean(k_range) + mean(k_comp)
    dec_path_ms = mean(k_doff) + mean(k_dec)
    roof["paths"] = {
        "compress_rel (range_kernel + compress_kernel)": {
            "ms": rel_ms, "bytes": 2 * field_bytes + size,
            "GB/s": (2 * field_bytes + size) / (rel_ms / 1e3) / 1e9,
            "frac": (2 * field_bytes + size) / (rel_ms / 1e3) / 1e9 / peak},
        "decompress (dec_offsets_kernel + decompress_kernel)": {
            "ms": dec_path_ms, "bytes": size + field_bytes,
            "GB/s": (size + field_bytes) / (dec_path_ms / 1e3) / 1e9,
            "frac": (size + field_bytes) / (dec_path_ms / 1e3) / 1e9 / peak},
    }
    # The whole calls (p50 of the call-timing pass): fz_compress with its
    # range pass, launches, result read-back and synchronisation against
    # 8 + 4/CR bytes per element; fz_decompress against 4/CR + 4.
    c50, d50 = percentile(call_c, 0.5), percentile(call_d, 0.5)
    roof["calls"] = {
        "fz_compress": {"ms_p50": c50, "bytes": 2 * field_bytes + size,
                        "GB/s": (2 * field_bytes + size) / (c50 / 1e3) / 1e9,
                        "frac": (2 * field_bytes + size) / (c50 / 1e3) / 1e9 / peak},
        "fz_decompress": {"ms_p50": d50, "bytes": size + field_bytes,
                          "GB/s": (size + field_bytes) / (d50 / 1e3) / 1e9,
                          "frac": (size + field_bytes) / (d50 / 1e3) / 1e9 / peak},
    }

    # the same compression as the paper's separate kernels (codes and
    # shuffled words through HBM): what fusing them saves on this GPU
    st_ms = []
    for _ in range(6):
        _, ssize, ms = codec.compress_staged_into(x_d, s_d, "rel", 1e-3, 3)
        st_ms.append(ms)
    assert ssize == size
    med = [statistics.median(m[k] for m in st_ms[1:]) for k in range(5)]
    # the same step with Listing 1's warp-ballot bitshuffle instead of the
    # register transpose (same stream)
    codec.set_staged_shuffle("ballot")
    bal_ms = []
    for _ in range(6):
        _, bsize, ms = codec.compress_staged_into(x_d, s_d, "rel", 1e-3, 3)
        bal_ms.append(ms[2])
    codec.set_staged_shuffle("register")
    assert bsize == size
    ablation = {"staged_kernel_ms": {"quantise": med[1], "shuffle_mark": med[2],
                                     "scan": med[3], "encode": med[4]},
                "staged_compress_ms": sum(med[1:]),
                "fused_compress_ms": mean(k_comp),
                "fusion_speedup": sum(med[1:]) / mean(k_comp),
                "shuffle_mark_ballot_ms": statistics.median(bal_ms[1:]),
                "shuffle_mark_register_ms": med[2]}

    # the whole-field Lorenzo variant (stream version 2) through the same
    # calls, timed by the library's call events: its stream size, and the
    # cost of its decompression (faces pass, cross-chunk scans, field pass)
    codec.set_call_timing(True)
    wc, wd = [], []
    for _ in range(6):
        _, wsize = codec.compress_into(x_d, s_d, "rel", 1e-3, 3, whole=True)
        wc.append(codec.call_times_ms()[0])
        codec.decompress_into(s_d, y_d, nbytes=wsize)
        wd.append(codec.call_times_ms()[1])
    codec.set_call_timing(False)
    ablation["whole_field_lorenzo"] = {
        "stream_bytes": wsize, "stream_bytes_chunked": size,
        "fz_compress_whole_ms_p50": statistics.median(wc[1:]),
        "fz_decompress_v2_ms_p50": statistics.median(wd[1:]),
        "fz_compress_ms_p50": c50, "fz_decompress_ms_p50": d50}

    # end to end through the host-buffer calls (pinned host memory)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(codec, x_h, cap, world, field_bytes, args, torch)

    cpu = None
    if rank == 0 and world >= 1 and not args.no_cpu_baseline:
        import oracle
        t_all, _ = cpu_oracle_round_trip(x_h, all_cores=True)
        slab = S // 2
        t_one, _ = cpu_oracle_round_trip(x_h[:slab].copy())
        cpu = {"value": 2 * field_bytes / t_all / 1e9, "unit": "GB/s",
               "cores": oracle.threads(), "kind": "oracle",
               "sample": f"the whole {S}^3 field, one compress+decompress, the oracle's "
                         "all-cores variant (OpenMP over points, tiles and chunks; "
                         "serial compaction)",
               "seconds": t_all, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "one_thread": {"value": 2 * 4 * x_h[:slab].size / t_one / 1e9,
                              "unit": "GB/s", "cores": 1, "seconds": t_one,
                              "sample": f"{S}x{S}x{slab} slab (half) of the same field, "
                                        "one compress+decompress, single-threaded"}}
    value = world * 2 * field_bytes / (ms_step / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.size == 512 else f"cosmo3d_{args.size}",
                       "desc": WORKLOAD_DESC.replace("512x512x512", f"{args.size}^3"),
                       "field_bytes": field_bytes, "eb_mode": "rel", "eb": 1e-3,
                       "l2": "inputs larger than L2 (512 MiB field), no flush",
                       "parallelism": f"{world} independent field(s), one per GPU"},
            "compress_gbs": field_bytes / (statistics.mean(comp_ms) / 1e3) / 1e9,
            "decompress_gbs": field_bytes / (statistics.mean(dec_ms) / 1e3) / 1e9,
            "compress_ms": {"p50": percentile(comp_ms, 0.5), "p99": percentile(comp_ms, 0.99)},
            "decompress_ms": {"p50": percentile(dec_ms, 0.5), "p99": percentile(dec_ms, 0.99)},
            "call_ms": {"fz_compress": {"p50": c50, "p99": percentile(call_c, 0.99)},
                        "fz_decompress": {"p50": d50, "p99": percentile(call_d, 0.99)},
                        "note": "library events at each call's entry and after its "
                                "read-back; compress_ms/decompress_ms above add the "
                                "Python binding's overhead"},
            "kernel_ms": {"range": mean(k_range), "compress": mean(k_comp),
                          "outliers": mean(k_out), "decompress_offsets": mean(k_doff),
                          "decompress": mean(k_dec)},
            "ratio": field_bytes / size, "stream_bytes": size,
            "roofline": roof, "ablation": ablation, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    codec.close()


def run_e2e(codec, x_h, cap, world, field_bytes, args, torch):
    xh_pin = torch.from_numpy(x_h).pin_memory()
    sh_pin = torch.empty(cap, dtype=torch.uint8).pin_memory()
    yh_pin = torch.empty(x_h.shape, dtype=torch.float32).pin_memory()
    xh_np, sh_np, yh_np = xh_pin.numpy(), sh_pin.numpy(), yh_pin.numpy()
    codec.set_profiling(False)
    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        s_np = codec.compress_host(xh_np, "rel", 1e-3, 3, out=sh_np)
        codec.decompress_host(s_np, out=yh_np)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s_np = codec.compress_host(xh_np, "rel", 1e-3, 3, out=sh_np)
        codec.decompress_host(s_np, out=yh_np)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": world * 2 * field_bytes / e2e_s / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": field_bytes + int(s_np.size),
           "d2h_bytes_per_step": int(s_np.size) + field_bytes,
           "ms_per_step": 1e3 * e2e_s}
    return e2e

def grf_on_device(torch, shape, beta, gen, dev):
    """Seeded Gaussian random field on the GPU (white noise shaped to power
    ~ k^beta, unit std): synthetic input only, made with torch FFTs."""
    noise = torch.randn(shape, generator=gen, device=dev)
    spec = torch.fft.rfftn(noise)
    k2 = None
    for i, n in enumerate(shape):
        f = torch.fft.rfftfreq(n, device=dev) if i == len(shape) - 1 else torch.fft.fftfreq(n, device=dev)
        view = [1] * len(shape)
        view[i] = -1
        t = f.view(view) ** 2
        k2 = t if k2 is None else k2 + t
    amp = k2.pow(beta / 4.0)
    amp.view(-1)[0] = 0.0
    g = torch.fft.irfftn(spec * amp, s=shape)
    g = (g - g.mean()) / g.std()
    return g.float().contiguous()


def run_batch(args, rank, world, local_rank):
    """The batched workload: 256 uneven 2-D/3-D fields (byte sizes
    log-uniform on 64 KiB..64 MiB, spectral slope U[-4,-2], relative bound
    per field from {1e-2,1e-3,1e-4}) compressed by one planned batch (one
    persistent launch per dimensionality, CUDA graph), against one
    fz_compress call per field on the same fields."""
    import torch

    import paper_2304_12557_gb300 as fz
    from paper_2304_12557_gb300 import build, fields

    if rank == 0:
        build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gen = torch.Generator(device=dev).manual_seed(4 + 1000 * rank)
    specs = fields.batch_shapes(256, 4)
    xs, outs = [], []
    for shape, ndim, beta, eb in specs:
        x = grf_on_device(torch, shape, beta, gen, dev)
        tiles = fz.stream_min_bytes(list(shape[::-1]), ndim) // 32
        outs.append(torch.empty(64 + 32 * tiles + 4096 * tiles + 65536, dtype=torch.uint8,
                                device=dev))
        xs.append(x)
    torch.cuda.synchronize()
    in_bytes = sum(4 * x.numel() for x in xs)
    codec = fz.Codec(local_rank)
    batch = fz.Batch(codec, [(x, o, "rel", eb, nd) for x, o, (_, nd, _, eb) in zip(xs, outs, specs)])
    tune = batch.autotune(reps=3)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        sizes, sts = batch.compress()
    assert all(s == fz.OK for s in sts), sts
    # a spot check: a few fields against their single-field streams
    for i in (0, 17, 101, 255):
        single = codec.compress(xs[i], mode="rel", eb=specs[i][3], ndim=specs[i][1])
        assert torch.equal(single, outs[i][: sizes[i]]), i
    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ
                           else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank]))
    sampler.start()                      # samples under load: untimed runs first
    t_load = time.time()
    while time.time() - t_load < 0.3:
        batch.compress()
    torch.cuda.synchronize()
    ev = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.compress()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    runs = [a.elapsed_time(b) for a, b in ev]
    # one launch sequence per field (fz_compress per field), same fields
    per = []
    for _ in range(max(2, min(args.steps, 5))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for x, o, (_, nd, _, eb) in zip(xs, outs, specs):
            codec.compress_into(x, o, "rel", eb, nd)
        e1.record(stream)
        per.append((e0, e1))
    torch.cuda.synchronize()
    per_ms = [a.elapsed_time(b) for a, b in per]
    ms = statistics.mean(runs)
    stream_bytes = int(sum(sizes))
    alg = 2 * in_bytes + stream_bytes           # range read + compress read + stream written
    peak, peak_kind = peaks()
    value = world * in_bytes / (ms / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": "batched compress GB/s of fp32 input (256 uneven fields, rel eb per field)",
            "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian random fields made on the GPU)",
            "config": {"workload": "batch256", "fields": len(xs), "input_bytes": in_bytes,
                       "ndim_mix": {"2": sum(1 for s in specs if s[1] == 2),
                                    "3": sum(1 for s in specs if s[1] == 3)},
                       "l2": "2.4 GB of inputs, larger than L2; no flush",
                       "parallelism": f"{world} independent batch(es), one per GPU",
                       "tuning": tune},
            "batch_ms": {"p50": percentile(runs, 0.5), "p99": percentile(runs, 0.99)},
            "per_field_launch": {"ms": statistics.mean(per_ms),
                                 "GB/s": in_bytes / (statistics.mean(per_ms) / 1e3) / 1e9},
            "speedup_vs_per_field": statistics.mean(per_ms) / ms,
            "ratio": in_bytes / stream_bytes, "stream_bytes": stream_bytes,
            "roofline": {"bound": "hbm", "kernel": "whole batch run", "achieved": alg / (ms / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": alg},
            "cpu_baseline": None, "e2e": None,
            # per run: range, prepare, compress (one per dimensionality), escapes
            "gpu_launches": args.steps * (3 + len({s[1] for s in specs})),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    codec.close()


def run_serve(args, rank, world, local_rank):
    """The served workload: Poisson arrivals swept over rates of 100 to 5000
    requests/s, half compress and half decompress, fields drawn as in the
    batched workload plus a 1 GiB 3-D field on 2% of the requests, relative
    bounds from {1e-2,1e-3,1e-4}; a 40 GB device pool.  Inputs and outputs
    are pinned host buffers; a client thread submits at the arrival times
    while another fetches the results in order.  Beside it, the baseline:
    the same arrivals served one request at a time, each by one host-buffer
    call (fz_compress_host / fz_decompress_host: copy in, one launch
    sequence for the field, copy out)."""
    import threading

    import numpy as np
    import torch

    import paper_2304_12557_gb300 as fz
    from paper_2304_12557_gb300 import build, fields

    if rank == 0:
        build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gen = torch.Generator(device=dev).manual_seed(5 + 1000 * rank)
    rng = np.random.default_rng(5 + 1000 * rank)
    ebs = [1e-2, 1e-3, 1e-4]
    lib = []                       # (host field, ndim, streams per eb, host outputs)
    codec = fz.Codec(local_rank)
    shapes = [(s, nd, beta) for s, nd, beta, _ in fields.batch_shapes(48, 5)]
    shapes.append(((1024, 512, 512), 3, -3.0))          # the 1 GiB field
    for shape, nd, beta in shapes:
        xd = grf_on_device(torch, shape, beta, gen, dev)
        xh = torch.empty(shape, dtype=torch.float32).pin_memory()
        xh.copy_(xd)
        streams = []
        for eb in ebs:
            s = codec.compress(xd, mode="rel", eb=eb, ndim=nd)
            sh = torch.empty(s.numel(), dtype=torch.uint8).pin_memory()
            sh.copy_(s)
            streams.append(sh)
        cap = max(int(sh.numel()) for sh in streams)
        outs = (np.empty(0), torch.empty(cap + (1 << 20), dtype=torch.uint8).pin_memory(),
                torch.empty(shape, dtype=torch.float32).pin_memory())
        lib.append((xh, nd, streams, outs))
        del xd
    torch.cuda.synchronize()
    lams = [100, 200, 500, 1000, 2000, 5000]

    def arrivals(lam):
        n = 5000                                         # 5000 requests per rate (50 s at 100/s)
        t_arr = np.cumsum(rng.exponential(1.0 / lam, n))
        kinds = rng.uniform(size=n) < 0.5                # True: compress
        big = rng.uniform(size=n) < 0.02
        which = np.where(big, len(lib) - 1, rng.integers(0, len(lib) - 1, n))
        eb_i = rng.integers(0, 3, n)
        return n, t_arr, kinds, which, eb_i

    def summarise(lam, n, t_arr, which, done_t):
        nbytes = np.array([4 * lib[w][0].numel() for w in which], dtype=np.float64)
        lat = np.array([done_t[i] - t_arr[i] for i in range(n)])
        big = np.asarray(which) == len(lib) - 1
        return {"rate_req_s": lam, "requests": n,
                "offered_GB_s": float(nbytes.sum() / t_arr[-1] / 1e9),
                "served_GB_s": float(nbytes.sum() / max(done_t) / 1e9),
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "p50_ms_without_1GiB": float(np.percentile(lat[~big], 50) * 1e3),
                "p99_ms_without_1GiB": float(np.percentile(lat[~big], 99) * 1e3),
                "p50_ms_1GiB": float(np.percentile(lat[big], 50) * 1e3) if big.any() else None}

    plans = {lam: arrivals(lam) for lam in lams}     # the same arrivals for both arms
    srv = fz.Server(local_rank, pool_bytes=40 << 30, max_batch=256)
    sweep = []
    for lam in lams:
        n, t_arr, kinds, which, eb_i = plans[lam]
        ids = [None] * n
        done_t = [0.0] * n
        parts = {"queue_ms": [], "launch_wait_ms": [], "gpu_ms": [], "launch_to_done_ms": [],
                 "fetch_ms": []}
        srv.stats(reset=True)
        t0 = time.perf_counter()
        ready = threading.Semaphore(0)

        def submit():
            for i in range(n):
                dt = t0 + t_arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                xh, nd, streams, _ = lib[which[i]]
                if kinds[i]:
                    ids[i] = srv.submit_compress(xh, "rel", ebs[eb_i[i]], nd)
                else:
                    ids[i] = srv.submit_decompress(streams[eb_i[i]])
                ready.release()

        th = threading.Thread(target=submit)
        th.start()
        for i in range(n):
            ready.acquire()
            _, _, _, outs = lib[which[i]]
            srv.wait(ids[i])
            inf = srv.info(ids[i])
            tf = time.perf_counter()
            srv.fetch(ids[i], out=(outs[1] if kinds[i] else outs[2]).numpy())
            done_t[i] = time.perf_counter() - t0
            parts["queue_ms"].append(inf["admit_ms"] - inf["submit_ms"])
            parts["launch_wait_ms"].append(inf["launch_ms"] - inf["admit_ms"])
            parts["gpu_ms"].append(inf["gpu_end_ms"] - inf["gpu_start_ms"])
            parts["launch_to_done_ms"].append(inf["done_ms"] - inf["launch_ms"])
            parts["fetch_ms"].append(1e3 * (done_t[i] - (tf - t0)))
        th.join()
        st = srv.stats()
        row = summarise(lam, n, t_arr, which, done_t)
        row.update({"server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"],
                    "failed": st["failed"],
                    "time_means_ms": {k: float(np.mean(v)) for k, v in parts.items()}})
        sweep.append(row)
    srv.close()

    # the baseline: one request at a time through the host-buffer calls
    base = []
    for lam in lams:
        n, t_arr, kinds, which, eb_i = plans[lam]
        done_t = [0.0] * n
        t0 = time.perf_counter()
        for i in range(n):
            dt = t0 + t_arr[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            xh, nd, streams, outs = lib[which[i]]
            if kinds[i]:
                codec.compress_host(xh.numpy(), "rel", ebs[eb_i[i]], nd, out=outs[1].numpy())
            else:
                codec.decompress_host(streams[eb_i[i]].numpy(), out=outs[2].numpy())
            done_t[i] = time.perf_counter() - t0
        base.append(summarise(lam, n, t_arr, which, done_t))
    codec.close()
    for row, b in zip(sweep, base):
        row["one_at_a_time"] = b
        row["served_vs_one_at_a_time"] = row["served_GB_s"] / b["served_GB_s"]
    best = max(sweep, key=lambda r: r["served_GB_s"])
    if rank == 0:
        line = {
            "metric": "served GB/s of fp32 input and p50/p99 latency (Poisson arrivals, 50/50 "
                      "compress/decompress)",
            "value": best["served_GB_s"], "unit": "GB/s", "n_gpus": world, "steps": len(lams),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian random fields, pinned host buffers)",
            "config": {"workload": "serve", "pool_bytes": 40 << 30, "max_batch": 256,
                       "fields": len(lib), "rel_eb": ebs, "big_field": "1024x512x512 (1 GiB)",
                       "baseline": "the same arrivals, one request at a time, one "
                                   "fz_compress_host / fz_decompress_host call each",
                       "parallelism": f"{world} independent server(s), one per GPU"},
            "sweep": sweep, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
        }
        print(json.dumps(line), flush=True)


def ssim_2d(torch, a, b, data_range):
    """Mean SSIM of two 2-D fields (8x8 box windows, the usual constants):
    an evaluation aid, computed with torch ops."""
    import torch.nn.functional as F
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    a = a[None, None].double()
    b = b[None, None].double()
    k = torch.ones(1, 1, 8, 8, dtype=torch.float64, device=a.device) / 64.0
    mu_a, mu_b = F.conv2d(a, k), F.conv2d(b, k)
    s_aa = F.conv2d(a * a, k) - mu_a ** 2
    s_bb = F.conv2d(b * b, k) - mu_b ** 2
    s_ab = F.conv2d(a * b, k) - mu_a * mu_b
    s = ((2 * mu_a * mu_b + c1) * (2 * s_ab + c2)) / ((mu_a ** 2 + mu_b ** 2 + c1) * (s_aa + s_bb + c2))
    return float(s.mean())


def run_quality(args, rank):
    """Rate-distortion of the synthetic fields (the paper's quality metrics,
    Sec. 4.2-4.3): compression ratio, bit rate, max |x - x'| / eb, PSNR
    (value range over RMSE) and SSIM (2-D: the field; 3-D: the mean over z
    slices) at the relative bounds 1e-2, 5e-3, 1e-3, 5e-4 and 1e-4 (Sec. 4.1)."""
    import torch

    import paper_2304_12557_gb300 as fz
    from paper_2304_12557_gb300 import build, fields

    if rank != 0:
        return
    build.build()
    dev = torch.device("cuda", 0)
    codec = fz.Codec(0)
    cases = [("bumps3d_64", fields.bumps3d(64)), ("climate2d_1800x3600", fields.climate2d()),
             ("cosmo3d_512", fields.cosmo3d(args.size))]
    rows = []
    for name, x_h in cases:
        x = torch.from_numpy(x_h).to(dev)
        vr = float(x.max() - x.min())
        for eb in (1e-2, 5e-3, 1e-3, 5e-4, 1e-4):
            s = codec.compress(x, mode="rel", eb=eb)
            y = codec.decompress(s).view(x.shape)
            info = fz.inspect(s[:64].cpu().numpy().tobytes())
            d = (x.double() - y.double())
            rmse = float(d.pow(2).mean().sqrt())
            if x.dim() == 2:
                ss = ssim_2d(torch, x, y, vr)
            else:
                ss = statistics.mean(ssim_2d(torch, x[z], y[z], vr)
                                     for z in range(0, x.shape[0], max(1, x.shape[0] // 16)))
            rows.append({"field": name, "rel_eb": eb, "ratio": 4 * x.numel() / s.numel(),
                         "bits_per_value": 8 * s.numel() / x.numel(),
                         "max_err_over_eb": float(d.abs().max()) / info["eb"],
                         "psnr_db": 20 * math.log10(vr / rmse) if rmse > 0 else float("inf"),
                         "ssim": ss, "nnz_block_fraction": info["nnz_blocks"] / (256 * info["n_tiles"]),
                         "outliers": info["n_outliers"]})
    # point-wise relative bounds through the log transform (Sec. 4.1's
    # particle data): sign words count towards the compressed size
    xp = torch.from_numpy(fields.particles1d(1 << 24)).to(dev)
    pw_rows = []
    for eps in (1e-2, 1e-3, 1e-4):
        y, signs = codec.pwrel_forward(xp)
        s = codec.compress(y, mode="abs", eb=fz.pwrel_bound(eps), ndim=1)
        xr = codec.pwrel_inverse(codec.decompress(s), signs)
        nz = xp != 0
        rel = ((xr.double() - xp.double()).abs()[nz] / xp.double().abs()[nz]).max().item()
        nbytes = s.numel() + signs.numel() * 4
        pw_rows.append({"field": "particles1d_16M", "pw_rel_eps": eps,
                        "ratio": 4 * xp.numel() / nbytes,
                        "bits_per_value": 8 * nbytes / xp.numel(),
                        "sign_bits_per_value": 32 * signs.numel() / xp.numel(),
                        "max_rel_err_over_eps": rel / eps,
                        "exact_zeros": bool((xr[~nz] == 0).all().item())})
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_f, t_i = [], []
    for _ in range(10):
        ev[0].record()
        y, signs = codec.pwrel_forward(xp)
        ev[1].record()
        codec.pwrel_inverse(y, signs)
        ev[2].record()
        torch.cuda.synchronize()
        t_f.append(ev[0].elapsed_time(ev[1]))
        t_i.append(ev[1].elapsed_time(ev[2]))
    codec.close()
    print(json.dumps({"metric": "rate-distortion of the synthetic fields (ratio, PSNR, SSIM)",
                      "value": None, "unit": None, "config": {"workload": "quality"},
                      "rows": rows, "pwrel_rows": pw_rows,
                      "pwrel_transform_ms": {"forward_p50": statistics.median(t_f),
                                             "inverse_p50": statistics.median(t_i),
                                             "elements": xp.numel(),
                                             "note": "forward includes its flag read-back"}}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="cosmo3d_512",
                    choices=["cosmo3d_512", "batch256", "serve", "quality", "cpu_baseline"],
                    help="cosmo3d_512: the single-field round trip (default); batch256: "
                         "256 uneven fields through one planned batch; serve: the request "
                         "server under Poisson arrivals; quality: rate-distortion report; "
                         "cpu_baseline: the CPU oracle timed per field and bound")
    ap.add_argument("--size", type=int, default=512,
                    help="edge of the cubic field (512 = the workload; smaller "
                         "sizes only for profiling captures)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as d
        torch.cuda.set_device(local_rank)
        d.init_process_group("nccl")
        dist = d
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.workload == "batch256":
        run_batch(args, rank, world, local_rank)
    elif args.workload == "serve":
        run_serve(args, rank, world, local_rank)
    elif args.workload == "quality":
        run_quality(args, rank)
    elif args.workload == "cpu_baseline":
        run_cpu_baseline_table(args, rank)
    else:
        run_ours(args, rank, world, local_rank, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
