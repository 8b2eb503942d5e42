#!/usr/bin/env python3
"""Benchmark of the B300 SZx codec (one JSON line on rank 0).

Workload: the 512^3 f32 Gaussian random field (power spectrum |k|^-5/3, 25% of
the volume zeroed in four 32-plane z-slabs), value-range relative bound 1e-3,
block 128.  One step = compress the field and decompress the stream (every
step of the hot path), with inputs resident in HBM; the field (512 MiB) is
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` is whole-job throughput in GB/s of input bytes (Eq. 2-3 of the paper:
N * b / T) per round trip; compress and decompress rates are reported beside
it.  On one GPU the line also carries the other configurations, each from its
own timed loop: `config3` (the 384^3 f64 field), `batch96` (96 mixed fields,
batched against per-field plain launches) and `serve` (Poisson requests,
continuous batching against a plain queue).  `cpu_baseline` and the reference
arm time the CPU oracle on the same fixed slice of the field, one process per
host core on disjoint block ranges (and one thread beside it).  With N > 1
(torchrun) every rank codes its own field (independent problems: weak
scaling, no collective on the data path).

Other workloads (--workload): batch96, serve, dump, grf384f64, blocksweep (b =
32 ... 1024 on the headline field) and relsweep (the headline field at rel
1e-2, 1e-3 and 1e-4, and its lognormal variant at 1e-3).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SZx compress/decompress GB/s and % HBM peak at rel-eb 1e-3; ratio; p99 ms"
SHAPE = (512, 512, 512)
SHAPE_RUN = list(SHAPE)  # --size changes the cube edge (profiling captures)
REL = 1e-3
BLOCK = 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def queue_ahead(stream, steps, host_us_per_step=150.0):
    """Hold the stream in a short clock-bounded spin (torch's own sleep kernel,
    before the start event) while the host queues every timed step, so that a
    host stall (another thread taking the interpreter lock, a sampler waking)
    cannot leave the GPU idle inside the timed region.  The timed work itself
    is unchanged."""
    import torch

    seconds = 1e-3 + steps * host_us_per_step * 1e-6
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(seconds * 2.032e9))  # cycles at the B300's top SM clock


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def clocks_once(gpu_index):
    """One nvidia-smi reading of the clocks and throttle reasons (not a
    sampling loop): for the serving arms, whose loop is bound by the host's
    CUDA calls, a sampler polling the driver during the run halved the
    throughput at saturation."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={ClockSampler.FIELDS}",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
        parts = [p.strip() for p in out.strip().splitlines()[0].split(",")]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return {"sm_mhz": float(parts[1]), "sm_max_mhz": float(parts[2]),
                "reasons": [n for n, f in zip(names, parts[5:9]) if f.lower() in ("active", "1", "yes")]}
    except Exception:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


SAMPLE_PLANES = 128  # the oracle's slice of the field: the first 128 z-planes (128 MiB at 512^3)


def _oracle_chunk(task):
    """One oracle process's share: compress and decompress values [lo, hi) of
    the shared slice `reps` times; returns its seconds (spawned worker)."""
    shm_name, n, lo, hi, eb, block, reps = task
    import time as _t
    from multiprocessing import shared_memory

    import numpy as np

    import oracle
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        part = np.array(np.ndarray((n,), dtype=np.float32, buffer=shm.buf)[lo:hi])
    finally:
        shm.close()
    oracle.lib()
    t0 = _t.perf_counter()
    for _ in range(reps):
        oracle.decompress(oracle.compress(part, eb, block))
    return _t.perf_counter() - t0


class OracleTimer:
    """The oracle (as it stands) on a fixed slice of the field: one thread, and
    one process per host core on disjoint block ranges (blocks are coded
    independently, Algorithm 1, so the ranges make the same streams as one
    pass).  Processes are spawned (CUDA is already initialised in this
    process) and kept for repeated measurements."""

    def __init__(self, x_host, eb):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        from multiprocessing import shared_memory

        import numpy as np
        plane = x_host.size // SHAPE_RUN[0]
        self.planes = min(SAMPLE_PLANES, SHAPE_RUN[0])
        self.n = self.planes * plane
        self.eb = eb
        self.shm = shared_memory.SharedMemory(create=True, size=self.n * 4)
        np.ndarray((self.n,), dtype=np.float32, buffer=self.shm.buf)[:] = x_host[:self.n]
        self.x = np.array(x_host[:self.n])
        self.cores = os.cpu_count() or 1
        # (an executor, not a Pool: a worker that fails is reported, not respawned)
        self.pool = ProcessPoolExecutor(self.cores, mp_context=mp.get_context("spawn"))
        # equal block-aligned ranges, one per process
        nb = -(-self.n // BLOCK)
        edges = [min(self.n, (nb * i // self.cores) * BLOCK) for i in range(self.cores + 1)]
        self.ranges = [(edges[i], edges[i + 1]) for i in range(self.cores) if edges[i + 1] > edges[i]]
        list(self.pool.map(_oracle_chunk, [(self.shm.name, self.n, lo, hi, eb, BLOCK, 1) for lo, hi in self.ranges]))

    def single_thread(self, reps=1):
        import oracle
        t_c = t_d = 0.0
        for _ in range(reps):
            t0 = time.perf_counter()
            s = oracle.compress(self.x, self.eb, BLOCK)
            t1 = time.perf_counter()
            oracle.decompress(s)
            t2 = time.perf_counter()
            t_c += t1 - t0
            t_d += t2 - t1
        b = self.n * 4 * reps
        return {"value": b / 1e9 / (t_c + t_d), "unit": "GB/s", "cores": 1,
                "compress_mbs": b / 1e6 / t_c, "decompress_mbs": b / 1e6 / t_d, "seconds": t_c + t_d}

    def all_cores(self, reps=6):
        t0 = time.perf_counter()
        busy = list(self.pool.map(_oracle_chunk, [(self.shm.name, self.n, lo, hi, self.eb, BLOCK, reps)
                                                 for lo, hi in self.ranges]))
        wall = time.perf_counter() - t0
        return {"value": self.n * 4 * reps / 1e9 / wall, "unit": "GB/s", "cores": len(self.ranges),
                "seconds": wall, "cpu_seconds": sum(busy)}

    def sample(self):
        return (f"the first {self.planes} z-planes of the field ({self.n * 4 >> 20} MiB, "
                f"{-(-self.n // BLOCK)} blocks): compress + decompress")

    def close(self):
        self.pool.shutdown()
        self.shm.close()
        self.shm.unlink()


def time_oracle(x_host, eb):
    """cpu_baseline: the oracle on the fixed slice, on every host core
    (`value`) and on one thread (`single_thread`)."""
    ot = OracleTimer(x_host, eb)
    try:
        one = ot.single_thread(reps=2)
        runs = [ot.all_cores() for _ in range(3)]
        allc = sorted(runs, key=lambda r: r["value"])[1]  # the median of three
    finally:
        ot.close()
    return {"value": allc["value"], "unit": "GB/s", "cores": allc["cores"], "kind": "oracle",
            "sample": ot.sample() + f", {allc['cores']} processes on disjoint block ranges",
            "cpu": cpu_model(), "single_thread": one, "all_cores": allc}


def max_over_ranks(ms, world, device):
    """The slowest rank's time (every rank gets it); a barrier precedes it in
    the caller.  With one rank, the value itself."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput_gbs(bytes_per_rank, steps, max_ms, world):
    """Whole-job GB/s: every rank codes its own field (weak scaling), so the
    job moves world * bytes_per_rank per step in the slowest rank's time."""
    return world * bytes_per_rank * steps / (max_ms * 1e-3) / 1e9


def kernel_sources_sha256():
    """Hash of the CUDA sources (names and bytes, sorted by path)."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2201_13020_b300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                   glob.glob(os.path.join(csrc, "*.h")))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def make_field(device, seed):
    from paper_2201_13020_b300 import inputs
    g = inputs.grf_3d(tuple(SHAPE_RUN), -5.0 / 3.0, seed=seed, device=device)
    g = inputs.zero_slabs(g, 0.25, 32, seed=seed)
    return g.reshape(-1).contiguous()


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import torch
    x = make_field("cuda" if torch.cuda.is_available() else "cpu", seed=2)
    from paper_2201_13020_b300 import inputs
    eb = inputs.rel_to_abs(x, REL)
    xh = x.cpu().numpy()
    del x
    # each step: the oracle on the same fixed slice as the cpu_baseline leg,
    # one process per host core on disjoint block ranges
    ot = OracleTimer(xh, eb)
    try:
        samples, secs = [], []
        for i in range(args.warmup + args.steps):
            r = ot.all_cores()
            if i >= args.warmup:
                samples.append(r["value"])
                secs.append(r["seconds"])
        one = ot.single_thread(reps=1)
    finally:
        ot.close()
    v = statistics.median(samples)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_block(world),
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": ot.cores, "kind": "oracle",
                             "sample": ot.sample() + f", {len(ot.ranges)} processes on disjoint block ranges",
                             "cpu": cpu_model(), "single_thread": one},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_batch96(args, rank, count=96):
    """Many fields: `count` fields, sizes log-uniform 256 KiB - 512 MiB, 70% f32 /
    30% f64, 1-D / 2-D / 3-D generators, REL from {1e-2, 1e-3, 1e-4}, block 128.
    Times the round trip three ways on the same data: per-field plain launches
    (two per field and direction), the batched plan (one persistent launch per
    (dtype, block) group, CTAs per SM autotuned), and the batched plan replayed
    from a CUDA graph; checks that batched and plain streams are identical.
    Returns the measurement as a dict."""
    import numpy as np
    import torch

    import paper_2201_13020_b300 as szx
    from paper_2201_13020_b300 import inputs
    t_start = time.perf_counter()
    fields = inputs.mixed_fields(count, 256 << 10, 512 << 20, seed=4 + rank, device="cuda")
    xs = [f[0] for f in fields]
    ebs = [inputs.rel_to_abs(x, rel) for x, rel, _ in fields]
    k = len(xs)
    in_bytes = sum(x.numel() * x.element_size() for x in xs)
    stream = torch.cuda.current_stream()
    code = [szx.SZX_F32 if x.dtype == torch.float32 else szx.SZX_F64 for x in xs]

    # per-field plain launches (the output buffers carry the scratch tail)
    p_out = [torch.empty(szx.compress_bound(x.numel(), c, BLOCK), dtype=torch.uint8, device="cuda")
             for x, c in zip(xs, code)]
    p_res = torch.zeros(2 * k, dtype=torch.int64, device="cuda")

    def plain_compress():
        for i in range(k):
            szx.compress_async(xs[i], ebs[i], BLOCK, p_out[i], p_res[2 * i:2 * i + 2])

    # the plan in its default shape (8 consumer warps, as many CTAs as fit)
    # and the plan the autotuner shaped
    fixed, f_out, f_res = szx.batch_compress(xs, ebs, BLOCK)
    batch, b_out, b_res = szx.batch_compress(xs, ebs, BLOCK)
    tuned_c = batch.autotune()

    plain_compress()
    batch.run()
    torch.cuda.synchronize()
    nb = p_res.cpu().numpy().reshape(-1, 2)
    bb = b_res.cpu().numpy().reshape(-1, 2)
    if (nb[:, 1] != 0).any() or (bb[:, 1] != 0).any() or not np.array_equal(nb[:, 0], bb[:, 0]):
        raise RuntimeError("batched and plain compression disagree on sizes or status")
    for i in range(k):
        if not torch.equal(p_out[i][:nb[i, 0]], b_out[i][:nb[i, 0]]):
            raise RuntimeError(f"field {i}: batched stream differs from the plain one")
    stream_bytes = int(nb[:, 0].sum())

    bufs = [b_out[i][:int(nb[i, 0])] for i in range(k)]
    headers = [szx.header(b) for b in bufs]
    ys = [torch.empty_like(x) for x in xs]
    st = torch.zeros(k, dtype=torch.int32, device="cuda")

    def plain_decompress():
        for i in range(k):
            szx.decompress_async(bufs[i], headers[i], ys[i], st[i:i + 1])

    dfixed, _, _ = szx.batch_decompress(bufs, headers)
    dbatch, d_ys, d_st = szx.batch_decompress(bufs, headers)
    tuned_d = dbatch.autotune()

    side = torch.cuda.Stream()
    graphs = []
    for b in (batch, dbatch):
        b.run(stream=side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            b.run(stream=side)
        graphs.append(g)

    arms = {
        "plain": (plain_compress, plain_decompress),
        "batched_fixed": (fixed.run, dfixed.run),
        "batched": (batch.run, dbatch.run),
        "batched_graph": (graphs[0].replay, graphs[1].replay),
    }
    times = {}
    for name, (fc, fd) in arms.items():
        for _ in range(args.warmup):
            fc()
            fd()
        torch.cuda.synchronize()
        # steps queued back to back (the host's launch time is part of each
        # arm's cost), events around each direction
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        for e in ev:
            e[0].record(stream)
            fc()
            e[1].record(stream)
            fd()
            e[2].record(stream)
        torch.cuda.synchronize()
        tc = sum(e[0].elapsed_time(e[1]) for e in ev)
        td = sum(e[1].elapsed_time(e[2]) for e in ev)
        times[name] = (tc / args.steps, td / args.steps)
    torch.cuda.synchronize()
    if int(st.abs().sum()) or int(d_st.abs().sum()):
        raise RuntimeError("decompression status not OK")
    for i in range(k):
        if not torch.equal(ys[i], d_ys[i]):
            raise RuntimeError(f"field {i}: batched decode differs from the plain one")

    def rates(ms):
        return {"compress_gbs": in_bytes / (ms[0] * 1e-3) / 1e9, "decompress_gbs": in_bytes / (ms[1] * 1e-3) / 1e9,
                "round_trip_gbs": in_bytes / ((ms[0] + ms[1]) * 1e-3) / 1e9, "compress_ms": ms[0],
                "decompress_ms": ms[1]}

    out = {name: rates(ms) for name, ms in times.items()}
    best = out["batched_graph"]
    peak, peak_kind = peaks()
    alg = in_bytes + stream_bytes
    for i in range(k):
        n_ = int(f_res[2 * i].item())
        if n_ != int(nb[i, 0]) or not torch.equal(f_out[i][:n_], b_out[i][:n_]):
            raise RuntimeError(f"field {i}: the fixed and the tuned plan wrote different streams")
    del fixed, dfixed, f_out

    # every shape of every compression group, timed alone (what the tuner
    # compared): consumer warps per CTA x CTAs per SM
    shapes = []
    for gi, g in enumerate(tuned_c):
        one_ms = {}
        for nw in (8, 4):
            for ctas in (2, 1):
                try:
                    batch.set_group(gi, ctas, nw)
                except szx.SzxError:
                    continue
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                batch.run()
                e[0].record(stream)
                for _ in range(5):
                    batch.run()
                e[1].record(stream)
                torch.cuda.synchronize()
                one_ms[f"{nw}warps_{ctas}ctas"] = e[0].elapsed_time(e[1]) / 5
        batch.set_group(gi, g["ctas_per_sm"], g["warps_per_cta"])
        shapes.append({"dtype": g["dtype"], "block": g["block"], "whole_plan_ms": one_ms})

    # block 0: the tuner also chooses b (64, 128 or 256) per dtype group; the
    # streams change with b, so they are checked by decoding them
    auto, a_out, a_res = szx.batch_compress(xs, ebs, 0)
    tuned_a = auto.autotune()
    ga = torch.cuda.CUDAGraph()
    auto.run(stream=side)
    torch.cuda.synchronize()
    with torch.cuda.graph(ga, stream=side):
        auto.run(stream=side)
    for _ in range(args.warmup):
        ga.replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(args.steps):
        ga.replay()
    ev[1].record(stream)
    torch.cuda.synchronize()
    a_ms = ev[0].elapsed_time(ev[1]) / args.steps
    ar = a_res.cpu().numpy().reshape(-1, 2)
    if (ar[:, 1] != 0).any():
        raise RuntimeError("block-0 batch: a stream's status is not OK")
    a_bufs = [a_out[i][:int(ar[i, 0])] for i in range(k)]
    adec, a_ys, a_st = szx.batch_decompress(a_bufs, [szx.header(b_) for b_ in a_bufs])
    adec.autotune()
    adec.run()
    torch.cuda.synchronize()
    if int(a_st.abs().sum()):
        raise RuntimeError("block-0 batch: decompression status not OK")
    for i in range(k):
        if float((a_ys[i].double() - xs[i].double()).abs().max()) > ebs[i]:
            raise RuntimeError(f"block-0 batch: field {i} exceeds its bound")
    a_bytes = int(ar[:, 0].sum())
    auto_block = {"compress_gbs": in_bytes / (a_ms * 1e-3) / 1e9, "compress_ms": a_ms,
                  "stream_bytes": a_bytes, "cr": in_bytes / a_bytes, "groups": tuned_a,
                  "vs_block128_cr": (in_bytes / a_bytes) / (in_bytes / stream_bytes)}
    del auto, adec, a_out, a_ys, ga
    res = {"workload": f"batch{k}_mixed_f32f64_256KiB-512MiB_block128", "fields": k, "input_bytes": in_bytes,
           "stream_bytes": stream_bytes, "cr": in_bytes / stream_bytes,
           "f64_fields": int(sum(c == szx.SZX_F64 for c in code)), "arms": out,
           "speedup_vs_plain": {"batched_fixed": out["batched_fixed"]["round_trip_gbs"] / out["plain"]["round_trip_gbs"],
                                "batched": out["batched"]["round_trip_gbs"] / out["plain"]["round_trip_gbs"],
                                "batched_graph": best["round_trip_gbs"] / out["plain"]["round_trip_gbs"]},
           "tuned_vs_fixed": out["batched"]["round_trip_gbs"] / out["batched_fixed"]["round_trip_gbs"],
           "compress_shapes": shapes,
           "block0": auto_block,
           "hbm_frac_algorithmic": {"compress": alg / (best["compress_ms"] * 1e-3) / 1e9 / peak,
                                    "decompress": alg / (best["decompress_ms"] * 1e-3) / 1e9 / peak,
                                    "peak": f"hbm_gbs {peak} of {peak_kind}"},
           "autotune": {"compress": tuned_c, "decompress": tuned_d},
           "steps": args.steps,
           # per step and plan: the run's clear kernel and one launch per group
           "gpu_launches": args.steps * (2 + len(tuned_c) + len(tuned_d)),
           "wall_s": time.perf_counter() - t_start}
    del graphs, batch, dbatch, b_out, d_ys, p_out, ys, xs, fields
    torch.cuda.empty_cache()
    return res


def run_batch96(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r = measure_batch96(args, rank)
    best = r["arms"]["batched_graph"]
    if rank == 0:
        line = {"metric": METRIC, "value": best["round_trip_gbs"] * world, "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": best["compress_ms"] + best["decompress_ms"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": r["workload"], "fields": r["fields"], "input_bytes": r["input_bytes"],
                           "stream_bytes": r["stream_bytes"], "cr": r["cr"], "f64_fields": r["f64_fields"],
                           "l2": "no flush: the batch (8 GB) exceeds the 126 MB L2",
                           "parallelism": f"replicas{world}"},
                "arms": r["arms"], "speedup_vs_plain": r["speedup_vs_plain"],
                "hbm_frac_algorithmic": r["hbm_frac_algorithmic"], "tuned_vs_fixed": r["tuned_vs_fixed"],
                "block0": r["block0"], "autotune": r["autotune"], "compress_shapes": r["compress_shapes"],
                "gpu_launches": r["gpu_launches"], "gpu": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_serve(args, rank, count, rate):
    """Serving: Poisson arrivals, 60% compress / 40% decompress of earlier
    resident streams, sizes log-uniform 64 KiB - 256 MiB; half the compress
    requests are complex f64 state vectors (unit-norm Gaussian, interleaved
    re/im, 2^k amplitudes with 2^k * 16 bytes nearest the drawn size), half
    f32 fields (the 1-D recipe); REL from {1e-2, 1e-3, 1e-4}; streams resident
    in a 120 GB pool.  Two arms on the same requests: one slot (a plain queue)
    and continuous batching (8 slots, overlapped on the device).  Returns the
    measurement as a dict."""
    import math

    import numpy as np
    import torch

    from paper_2201_13020_b300 import inputs, serve
    t_start = time.perf_counter()
    rng = np.random.default_rng(77 + rank)
    specs = []
    t = 0.0
    comp = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        if comp and rng.random() < 0.40:
            specs.append(("decompress", t, int(rng.choice(comp))))
            continue
        nbytes = math.exp(rng.uniform(math.log(64 << 10), math.log(256 << 20)))
        rel = float(rng.choice([1e-2, 1e-3, 1e-4]))
        if rng.random() < 0.5:
            k = int(round(math.log2(nbytes / 16)))
            specs.append(("compress", t, ("sv", 1 << max(12, min(24, k)), rel, i)))
        else:
            specs.append(("compress", t, ("f32", max(128, int(nbytes) // 4), rel, i)))
        comp.append(len(specs) - 1)
    data = {}
    for kind, _, a in specs:
        if kind == "compress":
            what, n, rel, seed = a
            x = (inputs.state_vector(n, seed=seed, device="cuda") if what == "sv"
                 else inputs.sinusoid_1d_torch(n, seed=seed, device="cuda"))
            data[seed] = (x, inputs.rel_to_abs(x, rel))
    torch.cuda.synchronize()

    def requests():
        out = []
        for kind, t, a in specs:
            if kind == "compress":
                x, eb = data[a[3]]
                out.append(serve.Request("compress", t, x=x, eb=eb, block=BLOCK))
            else:
                out.append(serve.Request("decompress", t, source=a))
        return out

    arms = {}
    # one long-lived 120 GB pool for both arms (a pool allocated or freed just
    # before a run slows the host's launches for a while); each arm first runs
    # the whole request list once untimed, then gives its streams back
    pool = torch.empty((120 << 30) + 256, dtype=torch.uint8, device="cuda")
    pool = pool[(-pool.data_ptr()) % 256:][:120 << 30]
    for name, slots in (("queue_1slot", 1), ("continuous_8slots", 8)):
        server = serve.Server(slots=slots, pool=pool)
        warm = requests()
        server.run(warm)
        for r in warm:
            if r.kind == "compress":
                server.release(r.offset, r.nbytes)
        reqs = requests()
        span = server.run(reqs)
        torch.cuda.synchronize()
        bad = [i for i, r in enumerate(reqs) if r.status != 0]
        if bad:
            raise RuntimeError(f"{len(bad)} requests failed, first {bad[0]} status {reqs[bad[0]].status}")
        lat = np.array([r.done_s - r.arrival for r in reqs]) * 1e3
        lat_c = np.array([r.done_s - r.arrival for r in reqs if r.kind == "compress"]) * 1e3
        lat_d = np.array([r.done_s - r.arrival for r in reqs if r.kind == "decompress"]) * 1e3
        total = sum(r.nbytes_in for r in reqs)
        arms[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "p50_compress_ms": float(np.percentile(lat_c, 50)),
                      "p99_compress_ms": float(np.percentile(lat_c, 99)),
                      "p50_decompress_ms": float(np.percentile(lat_d, 50)),
                      "p99_decompress_ms": float(np.percentile(lat_d, 99)),
                      "gbs": total / span / 1e9, "makespan_s": span, "input_bytes": total,
                      "max_in_flight": server.max_in_flight,
                      "resident_stream_bytes": int(sum(r.nbytes for r in reqs if r.kind == "compress"))}
        for r in reqs:
            if r.kind == "compress":
                server.release(r.offset, r.nbytes)
        server.close()
        del server, reqs
    del pool, data
    torch.cuda.empty_cache()
    # one reading of the clocks once both arms are done: the serving loop is
    # bound by the host's CUDA calls at saturation, and an nvidia-smi run
    # during or shortly before a timed run made those calls about twice as
    # slow (846-857 against 1,855-1,866 GB/s at 300,000 arrivals/s)
    clocks = clocks_once(torch.cuda.current_device())
    best = arms["continuous_8slots"]
    return {"workload": f"serve_poisson{rate:g}_req{count}_64KiB-256MiB_60c40d", "requests": count,
            "compress": sum(k == "compress" for k, _, _ in specs),
            "decompress": sum(k == "decompress" for k, _, _ in specs), "pool_bytes": 120 << 30,
            "arrival_rate_per_s": rate, "block": BLOCK, "gbs": best["gbs"], "p50_ms": best["p50_ms"],
            "p99_ms": best["p99_ms"], "speedup_vs_queue": best["gbs"] / arms["queue_1slot"]["gbs"],
            "arms": arms, "clocks_after": clocks, "wall_s": time.perf_counter() - t_start}


def run_serve(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    r = measure_serve(args, rank, args.requests, args.rate)
    best = r["arms"]["continuous_8slots"]
    if rank == 0:
        line = {"metric": METRIC, "value": best["gbs"], "unit": "GB/s", "n_gpus": world, "steps": 1, "warmup": 1,
                "ms_per_step": best["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64(state vectors)+f32", "data": "synthetic",
                "config": {"workload": r["workload"], "requests": r["requests"], "compress": r["compress"],
                           "decompress": r["decompress"], "pool_bytes": r["pool_bytes"],
                           "arrival_rate_per_s": r["arrival_rate_per_s"], "block": BLOCK,
                           "parallelism": f"replicas{world}"},
                "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "arms": r["arms"],
                "clocks": r["clocks_after"],
                "gpu": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    return 0


def run_dump(args, world, rank, local):
    """Compressed dump to a host file and load back (the 512^3 f32 field, rel
    1e-3), against a raw dump / load of the same values through the same path
    (device-to-host copy into pinned memory, file write; and the reverse)."""
    import tempfile

    import torch

    from paper_2201_13020_b300 import dump, inputs
    torch.cuda.set_device(local)
    x = make_field("cuda", seed=2 + rank)
    eb = inputs.rel_to_abs(x, REL)
    in_bytes = x.numel() * 4
    d = args.dump_dir or tempfile.gettempdir()
    path = os.path.join(d, f"szx_dump_{os.getpid()}.bin")
    raw_path = path + ".raw"
    chunk = 1 << 24  # 64 MiB of f32 per chunk

    def raw_dump():
        host = torch.empty(x.numel(), dtype=torch.float32, pin_memory=True)
        host.copy_(x)
        with open(raw_path, "wb") as f:
            f.write(memoryview(host.numpy()))

    def raw_load():
        host = torch.empty(x.numel(), dtype=torch.float32, pin_memory=True)
        with open(raw_path, "rb") as f:
            f.readinto(memoryview(host.numpy()))
        return host.cuda()

    res = {}
    try:
        for name, fn in (("szx_dump", lambda: dump.dump(x, eb, path, chunk_values=chunk)),
                         ("szx_load", lambda: dump.load(path)), ("raw_dump", raw_dump), ("raw_load", raw_load)):
            times = []
            for i in range(args.warmup + args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                if i >= args.warmup:
                    times.append(time.perf_counter() - t0)
            res[name] = {"gbs": in_bytes / statistics.median(times) / 1e9, "ms": 1e3 * statistics.median(times)}
        y = dump.load(path)
        e = float((y.double() - x.double()).abs().max())
        file_bytes = os.path.getsize(path)
    finally:
        for p_ in (path, raw_path):
            if os.path.exists(p_):
                os.remove(p_)
    if e > eb:
        raise RuntimeError(f"loaded values exceed the bound: {e} > {eb}")
    if rank == 0:
        line = {"metric": METRIC, "value": res["szx_dump"]["gbs"], "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["szx_dump"]["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "dump_grf512_f32_rel1e-3_chunk64MiB", "file_bytes": file_bytes,
                           "input_bytes": in_bytes, "cr": in_bytes / file_bytes, "dir": d,
                           "parallelism": f"replicas{world}"},
                "arms": res, "max_abs_error": e, "eb": eb, "gpu": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    return 0


def _sweep_row(x, eb, b, args):
    """Time compress_async / decompress_async of x at bound eb and block b
    (warm-up, then the median of the steps, queued as in the headline loop),
    check the decode against the bound, and return the row's rates, ratio,
    PSNR and block counts."""
    import torch

    import paper_2201_13020_b300 as szx
    from paper_2201_13020_b300 import metrics
    n = x.numel()
    stream = torch.cuda.current_stream()
    out = torch.empty(szx.compress_bound(n, szx.SZX_F32, b), dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    s0 = szx.compress(x, eb, b, out=out)
    nbytes = s0.numel()
    h = szx.header(out[:nbytes])
    y = torch.empty_like(x)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        szx.compress_async(x, eb, b, out, res)
        szx.decompress_async(out[:nbytes], h, y, st)
    torch.cuda.synchronize()
    # as in the headline loop: every timed step queued behind the clock-bounded
    # sleep, so that no host launch gap falls between a step's events
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    queue_ahead(stream, args.steps)
    for e in ev:
        e[0].record(stream)
        szx.compress_async(x, eb, b, out, res)
        e[1].record(stream)
        szx.decompress_async(out[:nbytes], h, y, st)
        e[2].record(stream)
    torch.cuda.synchronize()
    tc = [e[0].elapsed_time(e[1]) for e in ev]
    td = [e[1].elapsed_time(e[2]) for e in ev]
    if int(st.item()) or int(res[1].item()):
        raise RuntimeError(f"block {b}: status {int(res[1].item())}/{int(st.item())}")
    err = float((y.double() - x.double()).abs().max())
    if err > eb:
        raise RuntimeError(f"block {b}: error {err} > {eb}")
    nb = -(-n // b)
    peak, _ = peaks()
    alg = n * 4 + nbytes
    tcm, tdm = statistics.median(tc) * 1e-3, statistics.median(td) * 1e-3
    return {"compress_gbs": n * 4 / tcm / 1e9, "decompress_gbs": n * 4 / tdm / 1e9,
            "compress_us": tcm * 1e6, "decompress_us": tdm * 1e6,
            "hbm_frac_algorithmic": {"compress": alg / tcm / 1e9 / peak, "decompress": alg / tdm / 1e9 / peak},
            "cr": n * 4 / nbytes, "psnr_db": metrics.psnr(x, y),
            "constant_fraction": 1.0 - h.nonconst / nb, "raw_blocks": h.raw,
            "escalated_blocks": h.escalated}


def run_blocksweep(args, world, rank, local):
    """Block length sweep on the 512^3 f32 field at rel 1e-3 (Sec. V-A.2's
    study, Fig. 7, on synthetic data): per b, compress and decompress rates,
    compression ratio, Eq. 7 PSNR and the constant-block fraction; and the
    block length that block=0 picks."""
    import torch

    from paper_2201_13020_b300 import inputs, metrics
    torch.cuda.set_device(local)
    x = make_field("cuda", seed=2 + rank)
    eb = inputs.rel_to_abs(x, REL)
    rows = {b: _sweep_row(x, eb, b, args) for b in (32, 64, 128, 256, 512, 1024)}
    pick, sample_cr = metrics.choose_block(x, eb)
    if rank == 0:
        line = {"metric": METRIC, "value": rows[128]["compress_gbs"], "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "blocksweep_grf512_f32_rel1e-3", "parallelism": f"replicas{world}"},
                "blocks": rows, "block0_choice": pick, "block0_sample_cr": sample_cr,
                "gpu": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    return 0


def run_relsweep(args, world, rank, local):
    """The 512^3 f32 field at value-range bounds 1e-2, 1e-3 and 1e-4, and its
    lognormal variant (exp(1.5 g), the same zero slabs) at 1e-3, all at b =
    128: per case compress and decompress rates, the algorithmic HBM
    fractions, compression ratio, Eq. 7 PSNR and the block counts."""
    import torch

    from paper_2201_13020_b300 import inputs
    torch.cuda.set_device(local)
    rows = {}
    x = make_field("cuda", seed=2 + rank)
    for rel in (1e-2, 1e-3, 1e-4):
        rows[f"grf_rel{rel:g}"] = _sweep_row(x, inputs.rel_to_abs(x, rel), BLOCK, args)
    del x
    g = inputs.grf_3d(tuple(SHAPE_RUN), -5.0 / 3.0, seed=2 + rank, device="cuda")
    g = inputs.zero_slabs(inputs.lognormal(g), 0.25, 32, seed=2 + rank)
    x = g.reshape(-1).contiguous()
    del g
    rows["lognormal_rel0.001"] = _sweep_row(x, inputs.rel_to_abs(x, 1e-3), BLOCK, args)
    if rank == 0:
        line = {"metric": METRIC, "value": rows["grf_rel0.001"]["compress_gbs"], "unit": "GB/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "relsweep_grf512_f32_block128", "parallelism": f"replicas{world}"},
                "peak": "hbm_gbs %s of %s" % peaks(), "rows": rows,
                "gpu": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    return 0


def measure_f64(args, rank, rels=(1e-4, 1e-6), blocks=(128, 256)):
    """The f64 field: 384^3, spectrum |k|^-11/3 plus 1e-6 white noise; per REL
    and block: compress and decompress medians, rates, CR and the HBM fraction
    of the algorithmic bytes (input + stream).  Returns a dict of rows."""
    import torch

    import paper_2201_13020_b300 as szx
    from paper_2201_13020_b300 import inputs
    t_start = time.perf_counter()
    g = inputs.grf_3d((384, 384, 384), -11.0 / 3.0, seed=3 + rank, device="cuda", dtype=torch.float64)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(33 + rank)
    x = (g + 1e-6 * torch.randn(g.shape, generator=gen, device="cuda", dtype=torch.float64)).reshape(-1)
    del g
    n = x.numel()
    in_bytes = n * 8
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    rows = {}
    for rel in rels:
        eb = inputs.rel_to_abs(x, rel)
        for b in blocks:
            out = torch.empty(szx.compress_bound(n, szx.SZX_F64, b), dtype=torch.uint8, device="cuda")
            res = torch.zeros(2, dtype=torch.int64, device="cuda")
            nbytes = szx.compress(x, eb, b, out=out).numel()
            h = szx.header(out[:nbytes])
            y = torch.empty_like(x)
            st = torch.zeros(1, dtype=torch.int32, device="cuda")
            for _ in range(args.warmup):
                szx.compress_async(x, eb, b, out, res)
                szx.decompress_async(out[:nbytes], h, y, st)
            torch.cuda.synchronize()
            # the steps queued back to back, events around each kernel
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
            queue_ahead(stream, args.steps)
            for e in ev:
                e[0].record(stream)
                szx.compress_async(x, eb, b, out, res)
                e[1].record(stream)
                szx.decompress_async(out[:nbytes], h, y, st)
                e[2].record(stream)
            torch.cuda.synchronize()
            tc = [e[0].elapsed_time(e[1]) for e in ev]
            td = [e[1].elapsed_time(e[2]) for e in ev]
            if int(st.item()) or int(res[1].item()) or float((x - y).abs().max()) > eb:
                raise RuntimeError(f"rel {rel} block {b}: failed")
            mc, md = statistics.median(tc), statistics.median(td)
            alg = in_bytes + nbytes
            rows[f"rel{rel:g}_b{b}"] = {"compress_us": 1e3 * mc, "decompress_us": 1e3 * md,
                                         "compress_gbs": in_bytes / (mc * 1e-3) / 1e9,
                                         "decompress_gbs": in_bytes / (md * 1e-3) / 1e9,
                                         "cr": in_bytes / nbytes,
                                         "hbm_frac_compress": alg / (mc * 1e-3) / 1e9 / peak,
                                         "hbm_frac_decompress": alg / (md * 1e-3) / 1e9 / peak,
                                         "escalated_blocks": h.escalated, "raw_blocks": h.raw}
            del out, y
    del x
    torch.cuda.empty_cache()
    return {"workload": "grf384_f64_k-11/3_noise1e-6", "peak": f"hbm_gbs {peak} of {peak_kind}",
            "steps": args.steps, "rows": rows, "wall_s": time.perf_counter() - t_start}


def run_grf384f64(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    r = measure_f64(args, rank)
    if rank == 0:
        line = {"metric": METRIC, "value": r["rows"]["rel0.0001_b128"]["compress_gbs"], "unit": "GB/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": r["workload"], "peak": r["peak"], "parallelism": f"replicas{world}"},
                "rows": r["rows"], "gpu": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    return 0


def config_block(world):
    edge = SHAPE_RUN[0]
    return {"workload": f"grf{edge}_f32_k-5/3_zero-slabs25_rel1e-3_block128", "shape": list(SHAPE_RUN),
            "dtype": "f32", "block": BLOCK, "rel_eb": REL, "spectrum": "k^-5/3", "zero_slabs": 0.25,
            "l2": "no flush: the 512 MiB field and its stream exceed the 126 MB L2",
            "parallelism": f"replicas{world}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the config3 / batch96 / serve sub-objects")
    ap.add_argument("--batch-fields", type=int, default=96, help="fields of the batch96 sub-object")
    ap.add_argument("--serve-requests", type=int, default=600, help="requests of the serve sub-object")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--size", type=int, default=512, help="cube edge (default 512; smaller only for captures)")
    ap.add_argument("--workload", default="grf512", choices=["grf512", "batch96", "serve", "dump", "blocksweep", "relsweep", "grf384f64"],
                    help="grf512: the 512^3 f32 field (default); batch96: 96 mixed fields, batched vs plain; "
                         "serve: Poisson request mix through the serving loop; dump: compressed dump to a file")
    ap.add_argument("--dump-dir", default=None, help="dump: directory of the dump file (default: the temp dir)")
    ap.add_argument("--requests", type=int, default=600, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=30000.0, help="serve: mean arrivals per second")
    args = ap.parse_args()
    SHAPE_RUN[:] = [args.size] * 3
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "batch96":
        return run_batch96(args, world, rank, local)
    if args.workload == "serve":
        return run_serve(args, world, rank, local)
    if args.workload == "dump":
        return run_dump(args, world, rank, local)
    if args.workload == "blocksweep":
        return run_blocksweep(args, world, rank, local)
    if args.workload == "grf384f64":
        return run_grf384f64(args, world, rank, local)
    if args.workload == "relsweep":
        return run_relsweep(args, world, rank, local)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2201_13020_b300 as szx
    from paper_2201_13020_b300 import inputs

    x = make_field("cuda", seed=2 + rank)
    n = x.numel()
    eb = inputs.rel_to_abs(x, REL)
    cap = szx.compress_bound(n, szx.SZX_F32, BLOCK)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    y = torch.empty_like(x)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    # one synchronous round trip gives the header (the stream layout is
    # deterministic, so every later step writes the same bytes)
    s0 = szx.compress(x, eb, BLOCK, out=out)
    nbytes = s0.numel()
    h = szx.header(out[:nbytes])
    cr = n * 4 / nbytes

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    def step(events=None):
        if events:
            events[0].record(stream)
        szx.compress_async(x, eb, BLOCK, out, res)
        if events:
            events[1].record(stream)
        szx.decompress_async(out[:nbytes], h, y, status)
        if events:
            events[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        torch.cuda.profiler.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        queue_ahead(stream, args.steps)
        t0.record(stream)
        for i in range(args.steps):
            step(ev[i])
        t1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t0.elapsed_time(t1)
    comp_ms = [e[0].elapsed_time(e[1]) for e in ev]
    deco_ms = [e[1].elapsed_time(e[2]) for e in ev]
    step_ms = [c + d for c, d in zip(comp_ms, deco_ms)]
    r = res.cpu().tolist()
    if r[1] != 0 or int(status.item()) != 0 or r[0] != nbytes:
        raise RuntimeError(f"device status: compress {r}, decompress {int(status.item())}")
    total_ms = max_over_ranks(total_ms, world, "cuda")
    in_bytes = n * 4
    value = job_throughput_gbs(in_bytes, args.steps, total_ms, world)
    comp_gbs = in_bytes / (statistics.median(comp_ms) * 1e-3) / 1e9
    deco_gbs = in_bytes / (statistics.median(deco_ms) * 1e-3) / 1e9
    alg_bytes = in_bytes + nbytes  # read the field + write the stream (and the reverse)
    peak, peak_kind = peaks()
    comp_alg = alg_bytes / (statistics.mean(comp_ms) * 1e-3) / 1e9
    deco_alg = alg_bytes / (statistics.mean(deco_ms) * 1e-3) / 1e9
    dominant = "compress_kernel" if statistics.mean(comp_ms) >= statistics.mean(deco_ms) else "decompress_kernel"
    achieved = comp_alg if dominant == "compress_kernel" else deco_alg
    # ncu DRAM traffic per launch of the dominant kernel, when the recorded
    # capture was taken on the current kernel sources (else null)
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        if tj.get("sources_sha256") == kernel_sources_sha256() and args.size == 512:
            traffic = tj.get(dominant)
    except Exception:
        pass

    # end to end through the public calls with host buffers (pinned): every
    # step copies its input in, compresses, decompresses (with the header built
    # from the compress call's own result) and copies the values out.  Serial:
    # one step after the other.  Pipelined: step s+1's host-to-device copy runs
    # while step s's values are copied out (the link is full duplex); the
    # device never runs ahead of the data it needs.
    e2e = e2e_serial = None
    xd = yd = outs = None
    if args.e2e_steps > 0:
        xh = torch.empty(n, dtype=torch.float32, pin_memory=True)
        xh.copy_(x)
        yh = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        xd = [torch.empty_like(x) for _ in range(2)]
        yd = [torch.empty_like(x) for _ in range(2)]
        outs = [out, torch.empty_like(out)]
        # compress results land in pinned, device-visible memory
        resh = torch.zeros((2, 2), dtype=torch.int64, pin_memory=True)
        sth = torch.zeros(2, dtype=torch.int32, pin_memory=True)
        std = torch.zeros(2, dtype=torch.int32, device="cuda")
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            a = time.perf_counter()
            xd[0].copy_(xh, non_blocking=True)
            s_ = szx.compress(xd[0], eb, BLOCK, out=outs[0])
            szx.decompress(s_, out=yd[0])
            yh[0].copy_(yd[0], non_blocking=True)
            torch.cuda.synchronize()
            if i:
                times.append(time.perf_counter() - a)
        e2e_serial = {"value": in_bytes / statistics.median(times) / 1e9, "unit": "GB/s",
                      "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": in_bytes + 16 + 64 + 4}

        s_in, s_work, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_comp = [torch.cuda.Event() for _ in range(2)]
        ev_dec = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        k = max(4, args.e2e_steps * 3)
        hdr = szx.header(outs[0][:s_.numel()])

        def pipelined(steps):
            with torch.cuda.stream(s_in):
                xd[0].copy_(xh, non_blocking=True)
            ev_in[0].record(s_in)
            for st_ in range(steps):
                bi = st_ % 2
                s_work.wait_event(ev_in[bi])
                szx.compress_async(xd[bi], eb, BLOCK, outs[bi], resh[bi], stream=s_work)
                ev_comp[bi].record(s_work)
                if st_ + 1 < steps:
                    nb_ = (st_ + 1) % 2
                    # the next input reuses buffer nb_: its compression (step
                    # st_ - 1) finished before this step's host read below
                    with torch.cuda.stream(s_in):
                        xd[nb_].copy_(xh, non_blocking=True)
                    ev_in[nb_].record(s_in)
                ev_comp[bi].synchronize()
                nbytes_, status_ = (int(v) for v in resh[bi].tolist())
                if status_ != 0:
                    raise RuntimeError(f"e2e compress status {status_}")
                h_ = szx.SzxHeader()
                h_.block, h_.tile_blocks, h_.n, h_.dtype, h_.total_bytes = (BLOCK, hdr.tile_blocks, n,
                                                                            szx.SZX_F32, nbytes_)
                if st_ >= 2:
                    s_work.wait_event(ev_out[bi])  # yd[bi] has been copied out
                szx.decompress_async(outs[bi][:nbytes_], h_, yd[bi], std[bi:bi + 1], stream=s_work)
                ev_dec[bi].record(s_work)
                s_out.wait_event(ev_dec[bi])
                with torch.cuda.stream(s_out):
                    yh[bi].copy_(yd[bi], non_blocking=True)
                    sth[bi:bi + 1].copy_(std[bi:bi + 1], non_blocking=True)
                ev_out[bi].record(s_out)
            torch.cuda.synchronize()
            if int(sth.abs().sum()):
                raise RuntimeError("e2e decompress status not OK")

        pipelined(2)  # warm
        torch.cuda.synchronize()
        a = time.perf_counter()
        pipelined(k)
        dt = time.perf_counter() - a
        e2e = {"value": in_bytes * k / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": in_bytes + 16 + 4, "steps": k,
               "how": "pipelined: step s+1's input copy overlaps step s's output copy"}
        if not (torch.equal(yh[0], y.cpu()) and torch.equal(yh[1], y.cpu())):
            raise RuntimeError("e2e decode differs from the device-resident decode")

    # the other configurations, measured in the same run on one GPU: the f64
    # field, the batched form against per-field plain launches, and the
    # serving loop against a plain queue (their own timed loops; not part of
    # `value`)
    extras = {}
    if world == 1 and not args.no_extras:
        xh = x.cpu().numpy()
        del out, y, xd, yd, outs
        torch.cuda.empty_cache()
        extras["config3"] = measure_f64(args, rank, rels=(1e-4, 1e-6), blocks=(128,))
        extras["batch96"] = measure_batch96(args, rank, count=args.batch_fields)
        extras["serve"] = measure_serve(args, rank, count=args.serve_requests, rate=30000.0)
    else:
        xh = x.cpu().numpy() if rank == 0 else None

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base = time_oracle(xh, eb)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_block(world),
            "compress_gbs": comp_gbs, "decompress_gbs": deco_gbs, "cr": cr,
            "compress_ms_median": statistics.median(comp_ms), "decompress_ms_median": statistics.median(deco_ms),
            "p50_ms": statistics.median(step_ms),
            "p99_ms": float(np.percentile(step_ms, 99)),
            "hbm_frac_input": {"compress": comp_gbs / peak, "decompress": deco_gbs / peak},
            "hbm_frac_algorithmic": {"compress": comp_alg / peak, "decompress": deco_alg / peak},
            "roofline": {"kernel": dominant, "bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_kind": f"hbm_gbs of {peak_kind}", "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes},
            "cpu_baseline": cpu_base, "e2e": e2e, "e2e_serial": e2e_serial, "clocks": clocks.summary(),
            # per step: the workspace clear and the compression kernel, the
            # status clear and the decompression kernel
            "gpu_launches": 4 * args.steps,
            "stream": {"bytes": nbytes, "nonconst": h.nonconst, "raw": h.raw, "escalated": h.escalated,
                       "blocks": -(-n // BLOCK)},
            "gpu": torch.cuda.get_device_name(local),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
