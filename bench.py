#!/usr/bin/env python
"""BOA Constrictor round-trip throughput on one B300 (or N replicas).

Workload: a 64 MiB synthetic ATLAS-like jet table (row-major 5 x f32 rows,
Poisson(6) jets per event) cut into 4096 streams of 16 KB, compressed and
decompressed with a random-init Mamba predictor (d_model 256, 3 layers,
d_state 16, expand 2).  One step = compress all streams + decompress all
streams (the whole hot path); value = uncompressed MB (10^6 bytes) / step
time, inputs resident in HBM.  The L2 is flushed (a 256 MiB write) before
every timed step.

The headline form computes the projections with FP32 accuracy on the tensor
cores (3xTF32 split; everything else FP32), held to the same log-probability
bound as the plain FP32 CUDA-core form.  The other forms (plain FP32, BF16,
FP8) are reported beside it with their own accuracy against the oracle.
`--report precision` runs the 4 MB records subset through every form.

`--impl reference` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_2511_11337_b300 import synth  # noqa: E402

METRIC = "compress & decompress MB/s on 1 B300 at <=0.5% code-length gap vs FP64 oracle"
UNIT = "MB/s"
N_STREAMS, STREAM_LEN = 4096, 16384
WORKLOAD = "ATLAS-like jet table, 64 MiB as 4096 x 16 KB streams; Mamba d_model=256, 3 layers, d_state=16, expand=2 (1.45 M params)"
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
PREC = {"fp32": 0, "bf16": 1, "tf32x3": 2, "fp8": 3, "fp32_onchip": 0}


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of n independent streams for one rank."""
    lo = n * rank // world
    return lo, n * (rank + 1) // world


def reduce_max(value: float, dist, device) -> float:
    """Max over ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist, device) -> float:
    """Sum over ranks (the bytes the whole job processed)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def sources_sha256(paths) -> str | None:
    """One hash over the given source files, in order (None if one is missing)."""
    h = hashlib.sha256()
    for rel in paths:
        f = os.path.join(ROOT, rel)
        if not os.path.exists(f):
            return None
        h.update(rel.encode() + b"\0" + open(f, "rb").read())
    return h.hexdigest()


def traffic_for(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if none of the
    kernel's sources (its file and every header it includes) changed since
    the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    ent = t.get(kernel)
    srcs = ent.get("sources") if isinstance(ent, dict) else None
    if not srcs or sources_sha256(srcs) != ent.get("sources_sha256"):
        return None
    return ent


# ---------------------------------------------------------------- rooflines per phase

def unit_peaks(device: int) -> dict:
    """Rates of the units the phases are bound by, measured on this GPU with
    the library's microbenchmarks (boa_microbench, CUDA-event timed): MUFU
    ex2 results/s, FP32 FMA FLOP/s, L2 read GB/s, and dense tcgen05 rates
    (M 128, N 256, warp-issued) for TF32, BF16 and E4M3."""
    import ctypes as C
    from paper_2511_11337_b300._lib import check, load
    lib = load()

    def mb(test, kind=0, N=256, flags=0):
        r, a = C.c_double(), C.c_double()
        check(lib.boa_microbench(device, test, kind, 128, N, flags, C.byref(r), C.byref(a)))
        return r.value

    best = lambda f: max(f() for _ in range(3))
    return {"mufu_ex2_per_s": best(lambda: mb(0)), "ffma_tflops": best(lambda: mb(1)) / 1e12,
            "l2_read_gbs": best(lambda: mb(3)) / 1e9,
            "tf32_tflops": best(lambda: mb(4, 0, 256, 5)) / 1e12,      # A from TMEM, straight-line issue
            "bf16_tflops": best(lambda: mb(4, 1, 256, 4)) / 1e12,
            "e4m3_tflops": best(lambda: mb(4, 2, 256, 4)) / 1e12,
            "how": "boa_microbench: best of 3, CUDA events; tensor rates M 128 N 256 K 32 bytes per instruction, "
                   "one CTA per SM issuing back to back"}


def work_per_byte(shape) -> dict:
    """Algorithmic work per uncompressed byte of the predictor + coder path
    (one predicted byte per input byte)."""
    d, E, N, K, r, nl, F = (shape.d_model, shape.d_inner, shape.d_state, shape.d_conv, shape.dt_rank,
                            shape.n_layer, shape.d_model * shape.ffn_mult)
    # the tensor-core projections: in_proj, x_proj, out_proj, FFN, head
    # (dt_proj, 2 r E per layer, runs on the CUDA cores inside the scan)
    gemm = 2 * nl * (d * 2 * E + E * (r + 2 * N) + E * d + 2 * d * F) + 2 * d * 256
    # exp(Delta A) per (channel, state); softplus (ex2 + lg2), the conv's and
    # the gate's SiLU (ex2 + rcp each) per channel; softmax ex2 per symbol
    mufu = nl * (E * N + 6 * E) + 256
    # decode step, state in HBM: each layer reads and writes h (N x E) and
    # reads the conv window (K - 1 rows of E), writing one row of it
    state = nl * (2 * N * E * 4 + (K - 1) * E * 4 + E * 4)
    return {"gemm_flop": gemm, "mufu_ops": mufu, "decode_state_bytes": state}


def phase_rooflines(shape, precision: str, comp_mbps: float, dec_mbps: float, peaks: dict, hbm_gbs: float) -> dict:
    """Each phase's achieved rate against the roofs that bound it."""
    w = work_per_byte(shape)
    # tensor (or FP32 FMA) roof for the projections, in the form's own FLOPs
    # per FP32-equivalent FLOP: 3xTF32 issues three TF32 products
    if precision == "tf32x3":
        gemm_peak, gemm_src = peaks["tf32_tflops"] / 3.0, "measured TF32 rate / 3 (three TF32 products per FP32 product)"
    elif precision == "bf16":
        gemm_peak, gemm_src = peaks["bf16_tflops"], "measured BF16 rate"
    elif precision == "fp8":
        gemm_peak, gemm_src = peaks["e4m3_tflops"], "measured E4M3 rate"
    else:
        gemm_peak, gemm_src = peaks["ffma_tflops"], "measured FP32 FMA rate (CUDA cores)"
    gemm_roof_mbps = gemm_peak * 1e12 / w["gemm_flop"] / 1e6
    mufu_roof_mbps = peaks["mufu_ex2_per_s"] / w["mufu_ops"] / 1e6
    state_roof_mbps = hbm_gbs * 1e9 / w["decode_state_bytes"] / 1e6
    return {
        "work_per_byte": w,
        "compress": {"MBps": comp_mbps,
                     "tensor": {"roof_MBps": gemm_roof_mbps, "frac": comp_mbps / gemm_roof_mbps,
                                "achieved_tflops": comp_mbps * 1e6 * w["gemm_flop"] / 1e12, "peak_tflops": gemm_peak,
                                "peak_source": gemm_src},
                     "mufu": {"roof_MBps": mufu_roof_mbps, "frac": comp_mbps / mufu_roof_mbps,
                              "achieved_ops_per_s": comp_mbps * 1e6 * w["mufu_ops"],
                              "peak_ops_per_s": peaks["mufu_ex2_per_s"], "peak_source": "measured ex2 rate"}},
        "decompress": {"MBps": dec_mbps,
                       "hbm_state": {"roof_MBps": state_roof_mbps, "frac": dec_mbps / state_roof_mbps,
                                     "bytes_per_byte": w["decode_state_bytes"], "peak_gbs": hbm_gbs,
                                     "peak_source": "hbm_gbs (MEASURED_PEAKS.json)"},
                       "tensor": {"roof_MBps": gemm_roof_mbps, "frac": dec_mbps / gemm_roof_mbps},
                       "mufu": {"roof_MBps": mufu_roof_mbps, "frac": dec_mbps / mufu_roof_mbps}},
    }


# ---------------------------------------------------------------- oracle leg

def oracle_sample(streams: list[bytes], prefix: int):
    """Time the FP64 oracle (compress + decompress) on the first `prefix`
    bytes of each given stream, one OpenMP thread per stream."""
    from oracle import oracle as O
    path = os.path.join(tempfile.mkdtemp(), "paper.boaw")
    synth.make_model_file(path, synth.PAPER_SCALE, seed=2)
    m = O.Model(path)
    sample = [s[:prefix] for s in streams]
    threads = len(sample)
    t0 = time.perf_counter()
    comp = m.compress_batch(sample, n_threads=threads)
    dec, ok = m.decompress_batch(comp, [len(s) for s in sample], n_threads=threads)
    dt = time.perf_counter() - t0
    assert ok and dec == sample
    nbytes = sum(map(len, sample))
    return nbytes / 1e6 / dt, dt, nbytes, threads


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    buf = synth.atlas_workload(N_STREAMS, STREAM_LEN, seed=2000)
    streams = synth.split_equal(buf, N_STREAMS)[:cores]
    prefix = 2048
    for _ in range(args.warmup):
        oracle_sample(streams, 256)
    times, nb = [], 0
    for _ in range(args.steps):
        _, dt, nb, threads = oracle_sample(streams, prefix)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    v = nb / 1e6 / (ms / 1e3)
    sample = f"first {prefix} B of {len(streams)} of the 4096 streams ({nb} B), compress + decompress"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "streams": N_STREAMS, "stream_len": STREAM_LEN,
                   "parallelism": "host cores, one OpenMP thread per stream", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- precision forms

FORM_DESC = {"fp32": "plain FP32 on the CUDA cores", "tf32x3": "FP32-accurate 3xTF32 on the tensor cores",
             "bf16": "BF16 projections on the tensor cores", "fp8": "FP8 E4M3 projections on the tensor cores",
             "fp32_onchip": "plain FP32 on the CUDA cores; decompression by the on-chip persistent decoder "
                            "(one CTA per SM, two streams each, SSM state and conv windows in tensor memory)"}


def set_decoder(m, form):
    """The step-kernel decoder (model state in HBM) for every form but
    fp32_onchip, which takes the on-chip persistent decoder."""
    t = m.tuning()
    m.set_tuning(t["max_rows"], t["scan_variant"], t["decode_lanes"], decoder=int(form == "fp32_onchip"))


def form_accuracy(streams, forms, path, n_lp=4, lp_len=256, n_gap=16, gap_len=2048):
    """Against the FP64 oracle: max |d log2 p| over the first lp_len bytes of
    n_lp streams, and the code-length gap over gap_len-byte prefixes of n_gap
    streams (oracle on the host cores, one thread per stream)."""
    from oracle import oracle as O
    from paper_2511_11337_b300 import api
    om = O.Model(path)
    # streams spread evenly over the list (an uneven mix is not ordered by kind)
    pick = lambda n: [streams[i] for i in np.linspace(0, len(streams) - 1, min(n, len(streams))).astype(int)]
    lp_in = [s[:lp_len] for s in pick(n_lp) if len(s) >= 2]
    lp_ref = [om.logprobs(s) for s in lp_in]
    gap_in = [s[:gap_len] for s in pick(n_gap)]
    ref_total = sum(map(len, om.compress_batch(gap_in, n_threads=min(len(gap_in), os.cpu_count() or 1))))
    out = {}
    for f in forms:
        m = api.Model(path, precision=PREC[f])
        set_decoder(m, f)
        err = max(float(np.abs(m.logprobs(s) - r).max()) for s, r in zip(lp_in, lp_ref))
        comp = m.compress(gap_in)
        lossless = m.decompress(comp, [len(s) for s in gap_in]) == gap_in
        got = sum(map(len, comp))
        m.close()
        out[f] = {"form": FORM_DESC[f], "max_abs_dlog2p": err, "code_length_gap": (got - ref_total) / ref_total,
                  "sample_lossless": lossless,
                  "accuracy_sample": f"log2 p: first {lp_len} B of {len(lp_in)} streams; gap: first {gap_len} B of "
                                     f"{len(gap_in)} streams, both spread evenly over the workload's streams"}
    return out


def form_speed(form, path, d_in, in_off, d_out, out_off, d_dec, lens, stream, autotune=True, timed=3):
    """One warm-up and `timed` timed steps (mean) of another precision form
    (autotuned like the headline form)."""
    import torch
    from paper_2511_11337_b300 import api
    m = api.Model(path, cuda_stream=stream.cuda_stream, precision=PREC[form])
    if autotune:
        m.autotune(len(lens), int(max(lens)))
    set_decoder(m, form)
    total = int(in_off[-1])
    tcs, tds, lossless = [], [], True
    for k in range(1 + timed):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        a.record(stream)
        sizes = m.compress_device(d_in.data_ptr(), in_off, d_out.data_ptr(), out_off)
        b.record(stream)
        m.decompress_device(d_out.data_ptr(), out_off, lens, d_dec.data_ptr(), in_off, in_sizes=sizes)
        c.record(stream)
        torch.cuda.synchronize()
        lossless = lossless and bool(torch.equal(d_dec, d_in))
        if k >= 1:
            tcs.append(a.elapsed_time(b) / 1e3)
            tds.append(b.elapsed_time(c) / 1e3)
    m.close()
    tc, td = statistics.mean(tcs), statistics.mean(tds)
    return {"round_trip_MBps": total / 1e6 / (tc + td), "compress_MBps": total / 1e6 / tc,
            "decompress_MBps": total / 1e6 / td, "lossless": lossless, "timed_steps": timed,
            "round_trip_MBps_per_step": [total / 1e6 / (x + y) for x, y in zip(tcs, tds)]}


def run_precision_report(args):
    """The 4 MB records subset (256 streams x 16 KB, seeds 4000 + i) on the
    small records model (d_model 64, 2 layers) through every form: code-length
    gap on the whole subset and max |d log2 p| on 16 x 1 KB, against the FP64
    oracle, and round-trip MB/s on the GPU."""
    import torch
    rank, _, local = env_rank()
    if rank != 0:                                   # a report: rank 0 alone under torchrun
        return
    torch.cuda.set_device(local)
    from oracle import oracle as O
    from paper_2511_11337_b300 import api
    path = synth.make_model_file(os.path.join(tempfile.mkdtemp(), "tiny.boaw"), synth.TINY, seed=1)
    streams = synth.records_workload(256, 16384, seed_base=4000)
    om = O.Model(path)
    t0 = time.perf_counter()
    ref = om.compress_batch(streams, n_threads=os.cpu_count() or 1)
    t_oracle = time.perf_counter() - t0
    ref_total = sum(map(len, ref))
    lp_ref = [om.logprobs(s[:1024]) for s in streams[:16]]
    total = sum(map(len, streams))
    rows = {}
    for f in ("fp32", "tf32x3", "bf16", "fp8"):
        m = api.Model(path, precision=PREC[f])
        comp = m.compress(streams)
        ok = m.decompress(comp, [len(s) for s in streams]) == streams
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        comp = m.compress(streams)
        m.decompress(comp, [len(s) for s in streams])
        dt = time.perf_counter() - t0
        err = max(float(np.abs(m.logprobs(s[:1024]) - r).max()) for s, r in zip(streams[:16], lp_ref))
        got = sum(map(len, comp))
        rows[f] = {"form": FORM_DESC[f], "lossless": ok, "compressed_bytes": got,
                   "bits_per_byte": 8 * got / total, "code_length_gap": (got - ref_total) / ref_total,
                   "max_abs_dlog2p": err, "round_trip_MBps_host_api": total / 1e6 / dt}
        m.close()
    print(json.dumps({"report": "precision forms", "workload": "records subset, 256 x 16 KB (seeds 4000+i), "
                      "model d_model 64, 2 layers", "oracle_bits_per_byte": 8 * ref_total / total,
                      "oracle_s": t_oracle, "forms": rows}))


# ---------------------------------------------------------------- GPU leg

def run_boa(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2511_11337_b300 import api

    tmpd = tempfile.mkdtemp()
    path = synth.make_model_file(os.path.join(tmpd, "paper.boaw"), synth.PAPER_SCALE, seed=2)
    # The job is world x 64 MiB of independent streams; each rank compresses
    # its contiguous share (weak scaling, no data-path collective).
    lo, hi = shard_range(world * args.streams, rank, world)
    if args.workload == "mixed":
        # an uneven mix of ATLAS-like and CMS-like streams (log-uniform
        # 1 KB - 1 MB), each cut into 16 KB chunks as the container stores
        # it (a chunk is a coder stream)
        src = synth.mixed_workload(args.streams, seed=3000 + lo)
        streams = [s[i:i + args.stream_len] for s in src for i in range(0, len(s), args.stream_len)]
    else:
        buf = synth.atlas_workload(args.streams, args.stream_len, seed=2000 + lo // args.streams)
        streams = synth.split_equal(buf, args.streams)[: hi - lo]
    total = sum(map(len, streams))

    stream = torch.cuda.Stream()
    prec = PREC[args.precision]
    model = api.Model(path, device=local, cuda_stream=stream.cuda_stream, max_rows=args.max_rows, precision=prec)
    flat, in_off = api.pack(streams)
    lens = np.diff(in_off)
    out_off = api.compressed_slot_offsets(lens)
    d_in = torch.from_numpy(flat.copy()).cuda()
    d_out = torch.zeros(int(out_off[-1]), dtype=torch.uint8, device="cuda")
    d_dec = torch.zeros(total, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step(mid=None):
        sizes = model.compress_device(d_in.data_ptr(), in_off, d_out.data_ptr(), out_off)
        n1 = model.last_launch_count
        if mid is not None:
            mid.record(stream)
        model.decompress_device(d_out.data_ptr(), out_off, lens, d_dec.data_ptr(), in_off, in_sizes=sizes)
        return sizes, n1 + model.last_launch_count

    tuning = model.autotune(len(streams), int(np.median(lens))) if args.autotune else None
    if args.decode_lanes is not None or args.scan_variant is not None:
        t = model.tuning()
        model.set_tuning(t["max_rows"], t["scan_variant"] if args.scan_variant is None else args.scan_variant,
                         t["decode_lanes"] if args.decode_lanes is None else args.decode_lanes, t["decoder"])
        tuning = dict(tuning or {}, **model.tuning(), overridden=True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.warmup:
        assert torch.equal(d_dec, d_in), "round trip failed in warm-up"

    # timed region
    stride = 8
    model.profile(True, decode_step_stride=stride)
    model.profile_reset()
    evs = []
    launches = 0
    sizes = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            mid = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sizes, n = step(mid)
            b.record(stream)
            evs.append((a, mid, b))
            launches += n
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    model.profile(False)
    prof = model.profile_read()
    prof_steps = model.profile_steps()
    ms = statistics.mean(a.elapsed_time(b) for a, _, b in evs)
    # the phases as they ran (decode lanes overlap, so the per-class kernel
    # times below add up to more than the decompression phase)
    phase_ms = {"compress": round(statistics.mean(a.elapsed_time(c) for a, c, _ in evs), 1),
                "decompress": round(statistics.mean(c.elapsed_time(b) for _, c, b in evs), 1)}
    job_bytes = reduce_sum(float(total), dist, "cuda") if dist else float(total)
    if dist:
        ms = reduce_max(ms, dist, "cuda")
        dist.barrier()
    assert torch.equal(d_dec, d_in), "round trip failed in timed region"
    comp_total = int(np.sum(sizes))

    # end to end through the host API (pinned staging, H2D, compute, D2H)
    e2e = None
    if args.e2e_steps > 0:
        e2e_times = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            comp = model.compress(streams)
            dec = model.decompress(comp, [len(s) for s in streams])
            e2e_times.append(time.perf_counter() - t0)
        assert dec == streams
        e2e_comp = sum(map(len, comp))
        e2e_s = statistics.mean(e2e_times)
        if dist:
            e2e_s = reduce_max(e2e_s, dist, "cuda")      # the job ends with its slowest rank
        e2e = {"value": job_bytes / 1e6 / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": total + e2e_comp, "d2h_bytes_per_step": e2e_comp + total}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    value = job_bytes / 1e6 / (ms / 1e3)
    peaks, peak_src = measured_peaks()
    # Per-(phase, class) device time per step: compression launches are all
    # timed; of the decode steps (CUDA graphs of 32) one eager step per graph
    # launch is timed, so scale by all steps / timed steps.
    est = {}
    for phase, d in prof.items():
        n_timed, n_all = prof_steps[phase]
        for k, v in d.items():
            scale = (n_all / n_timed if n_timed else 0.0) / args.steps
            est[(phase, k)] = dict(v, ms_step=v["ms"] * scale)
    step_est = sum(v["ms_step"] for v in est.values())
    dom = max(est, key=lambda k: est[k]["ms_step"]) if est else None
    roof = None
    if dom:
        p = est[dom]
        name = f"{dom[1]} ({dom[0]})"
        if dom[1].startswith("gemm") and args.precision in ("bf16", "tf32x3", "fp8"):
            achieved = p["flops"] / (p["ms"] / 1e3) / 1e12
            # a contraction's peak for its own dtype: the measured BF16 rate
            # times the nominal dense ratio (FP8 4.5/2.25, TF32 1.1/2.25; the
            # 3xTF32 form issues three TF32 products per FP32 product)
            ratio = {"bf16": 1.0, "fp8": 2.0, "tf32x3": (1.1 / 2.25) / 3.0}[args.precision]
            pk = peaks["bf16_tflops_sustained"] * ratio
            roof = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                    "kernel": name,
                    "peak_source": f"bf16_tflops_sustained ({peak_src}) x {ratio:.4f} for {args.precision}"}
        elif dom[1].startswith("gemm"):
            achieved = p["flops"] / (p["ms"] / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS, "kernel": name,
                    "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x 2.032 GHz (FP32 FFMA pipe)"}
        else:
            achieved = p["bytes"] / (p["ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "kernel": name, "peak_source": f"hbm_gbs ({peak_src})"}
        tr = traffic_for(f"{dom[0]}:{dom[1]}")
        roof["avg_launch_ms"] = p["ms"] / p["launches"]
        roof["algorithmic_per_launch"] = (p["flops"] if dom[1].startswith("gemm") else p["bytes"]) / p["launches"]
        roof["traffic"] = tr["bytes_per_launch"] if tr else None
        if tr and tr.get("algorithmic_per_launch"):
            # the capture's launch may process another number of slots: its
            # DRAM bytes scaled by the ratio of algorithmic bytes (the state
            # traffic grows in proportion to the slots)
            scale = roof["algorithmic_per_launch"] / tr["algorithmic_per_launch"]
            if abs(scale - 1.0) > 1e-6:
                roof["traffic"] = tr["bytes_per_launch"] * scale
                roof["traffic_scaled_from"] = {"bytes_per_launch": tr["bytes_per_launch"],
                                               "algorithmic_per_launch": tr["algorithmic_per_launch"],
                                               "scale": scale}
    if roof is not None and world == 1:
        try:
            up = unit_peaks(local)
            roof["unit_peaks_measured"] = up
            roof["phases"] = phase_rooflines(
                synth.PAPER_SCALE, args.precision, total / 1e6 / (phase_ms["compress"] / 1e3),
                total / 1e6 / (phase_ms["decompress"] / 1e3), up, peaks["hbm_gbs"])
        except Exception as e:                       # a report, never a reason to lose the bench line
            roof["phases"] = {"error": str(e)}
    breakdown = {f"{ph}:{k}": {"launches_timed": v["launches"], "ms_per_step": round(v["ms_step"], 2),
                               "share": round(v["ms_step"] / step_est, 4) if step_est else None}
                 for (ph, k), v in sorted(est.items(), key=lambda kv: -kv[1]["ms_step"])}
    kernel_ms = {ph: round(sum(v["ms_step"] for (p2, _), v in est.items() if p2 == ph), 1)
                 for ph in ("compress", "decompress")}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v_cpu, dt, nb, threads = oracle_sample(streams[:cores], args.cpu_prefix)
        one = max(args.cpu_prefix // 4, 2)
        v_1, dt_1, nb_1, _ = oracle_sample(streams[:1], one)
        cpu = {"value": v_cpu, "unit": UNIT, "cores": threads, "kind": "oracle", "nproc": cores,
               "sample": f"first {args.cpu_prefix} B of {threads} of the 4096 streams ({nb} B), compress + decompress, {dt:.1f} s",
               "single_thread": {"value": v_1, "unit": UNIT,
                                 "sample": f"first {one} B of stream 0, one thread, {dt_1:.1f} s"}}

    forms = {}
    if world == 1:
        # the headline form's accuracy against the oracle on a sample is
        # always reported; the other forms' accuracy and speed on request
        names = [f for f in args.forms.split(",") if f and f != args.precision]
        acc = form_accuracy(streams, [args.precision] + names, path)
        forms[args.precision] = dict(acc[args.precision], round_trip_MBps=value,
                                     compress_MBps=total / 1e6 / (phase_ms["compress"] / 1e3),
                                     decompress_MBps=total / 1e6 / (phase_ms["decompress"] / 1e3))
        model.close()
        for f in names:
            forms[f] = dict(acc[f], **form_speed(f, path, d_in, in_off, d_out, out_off, d_dec, lens, stream,
                                                 args.autotune))

    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32x3": "f32 (projections as 3xTF32 on tensor cores)",
                  "bf16": "bf16 projections, f32 elsewhere", "fp8": "e4m3 projections, f32 elsewhere"}[args.precision],
        "data": "synthetic",
        "config": {"workload": (f"uneven mix: {args.streams} streams of log-uniform 1 KB-1 MB, ATLAS-like or "
                                f"CMS-like at random, cut into {len(streams)} chunks of at most {args.stream_len} B; "
                                "same model") if args.workload == "mixed" else
                   WORKLOAD if (args.streams, args.stream_len) == (N_STREAMS, STREAM_LEN) else
                   f"reduced: {args.streams} x {args.stream_len} B of the jet table, same model",
                   "streams": args.streams, "stream_len": args.stream_len, "bytes_per_gpu": total,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed (256 MiB write) before every timed step", "autotuned": tuning},
        "compression_ratio": total / comp_total,
        "compressed_bytes": comp_total,
        # the paper's space-saving rate (original - compressed) / time, here per round trip
        "sigma_ssr_MBps": world * (total - comp_total) / 1e6 / (ms / 1e3),
        "wall_s_timed": t_wall,
        "e2e": e2e,
        "gpu_launches": launches,
        "phase_ms_per_step": phase_ms,
        "kernel_ms_sum_per_step": kernel_ms,
        "compress_MBps": total / 1e6 / (phase_ms["compress"] / 1e3) if phase_ms["compress"] else None,
        "decompress_MBps": total / 1e6 / (phase_ms["decompress"] / 1e3) if phase_ms["decompress"] else None,
        "roofline": roof,
        "kernel_breakdown": breakdown,
        "profiled_steps": {ph: {"timed": a, "all": b} for ph, (a, b) in prof_steps.items()},
        "cpu_baseline": cpu,
        "precision_forms": forms,
        "clocks": clocks,
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_stream_report(args):
    """The streaming pipeline (boa_stream_*) on the 64 MiB jet table: bytes
    pushed from host memory in 4 MiB pieces, one .boa shard per set of
    --set-chunks x 16 KB chunks (each set compressed while the next one
    fills and pre-loads), then boa_unpack_shards back to host memory; and
    boa_pack / boa_unpack of the same bytes as one container, for
    comparison.  Host clock around the synchronous calls (host buffers at
    both ends); rank 0 only."""
    import torch
    rank, _, local = env_rank()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_2511_11337_b300 import api
    path = synth.make_model_file(os.path.join(tempfile.mkdtemp(), "paper.boaw"), synth.PAPER_SCALE, seed=2)
    buf = synth.atlas_workload(args.streams, args.stream_len, seed=2000)
    model = api.Model(path, device=local, precision=PREC[args.precision], max_rows=args.max_rows)
    per = args.set_chunks
    tuned = model.autotune(per, args.stream_len) if args.autotune else None
    piece = 4 << 20

    def streamed(data):
        t0 = time.perf_counter()
        with api.Stream(model, args.stream_len, per) as st:
            for i in range(0, len(data), piece):
                st.push(data[i:i + piece])
            st.finish()
            blob = st.read()
            stats = st.stats()
        t1 = time.perf_counter()
        out = model.unpack_shards(blob)
        t2 = time.perf_counter()
        assert out == data
        return t1 - t0, t2 - t1, len(blob), stats

    def packed(data):
        t0 = time.perf_counter()
        box = model.pack(data, args.stream_len)
        t1 = time.perf_counter()
        assert model.unpack(box) == data
        return t1 - t0, time.perf_counter() - t1

    for _ in range(args.warmup):
        streamed(buf[:2 * per * args.stream_len])
    runs = [streamed(buf) for _ in range(args.steps)]
    tc = statistics.mean(r[0] for r in runs)
    td = statistics.mean(r[1] for r in runs)
    pk = [packed(buf) for _ in range(max(1, args.steps // 2))]
    pc, pd = statistics.mean(r[0] for r in pk), statistics.mean(r[1] for r in pk)
    mb = len(buf) / 1e6
    print(json.dumps({
        "report": "streaming pipeline", "metric": "streamed compress & decompress MB/s on 1 B300, host buffers at both ends",
        "value": mb / (tc + td), "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}; pushed in 4 MiB pieces, sets of {per} x {args.stream_len} B "
                               f"({len(buf) // (per * args.stream_len)} shards)", "autotuned": tuned},
        "compress_MBps": mb / tc, "decompress_MBps": mb / td, "compression_ratio": len(buf) / runs[-1][2],
        "sets": runs[-1][3]["sets"], "preloaded_sets": runs[-1][3]["preloaded"],
        "pack_unpack_MBps": mb / (pc + pd), "pack_MBps": mb / pc, "unpack_MBps": mb / pd,
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="boa", choices=["boa", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--streams", type=int, default=N_STREAMS)
    ap.add_argument("--stream-len", type=int, default=STREAM_LEN)
    ap.add_argument("--workload", default="jet", choices=["jet", "mixed", "stream"],
                    help="jet: the benchmark's 64 MiB jet table; mixed: an uneven ATLAS/CMS mix of log-uniform 1 KB-1 MB "
                         "streams (--streams sources); stream: the jet table through the streaming pipeline (a report)")
    ap.add_argument("--set-chunks", type=int, default=1024, help="chunks per streaming set (--workload stream)")
    ap.add_argument("--max-rows", type=int, default=0)
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "bf16", "tf32x3", "fp8"])
    ap.add_argument("--forms", default="fp32,fp32_onchip,bf16,fp8",
                    help="other precision forms to report ('' for none); fp32_onchip: the FP32 form decoded by "
                         "the on-chip persistent decoder")
    ap.add_argument("--report", default="", choices=["", "precision"])
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--decode-lanes", type=int, default=None, help="override the tuned decode lane count")
    ap.add_argument("--scan-variant", type=int, default=None, help="override the tuned decode scan kernel")
    ap.add_argument("--cpu-prefix", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.report == "precision":
        run_precision_report(args)
    elif args.workload == "stream":
        run_stream_report(args)
    else:
        run_boa(args)


if __name__ == "__main__":
    main()
