#!/usr/bin/env python3
"""Benchmark of the RANLUX++ hot path on GB300: the 2^20-stream workload.

One step = the whole hot path over 2^20 independent streams at luxury p = 2048:
  1. rlxpp_seed: stream i restarts at the seed-1 state skipped by i 2^96 advances
     (exponentiation by squaring over the power table, Sec. 2.4);
  2. rlxpp_draw_f64: 1024 doubles per stream written to HBM (8 GiB);
  3. rlxpp_draw_f64_sum_hist: 4096 more doubles per stream consumed in the kernel by an
     exact sum and a 256-bin histogram (no output traffic; the consumer of the paper's
     GPU benchmark, Sec. 4.2).
That is 5120 doubles and 426 LCG advances per stream per step.  Every step writes 8 GiB,
more than the 129 MB L2, so no explicit flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead (the
plain recurrence in C on the host cores, over a bounded sample of the same workload).
Under torchrun each rank runs its own disjoint range of streams (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LCG advances/s and random doubles/s on 1 GB300 (bit-exact), % of INT/IMMA roofline"
UNIT = "doubles/s"
N_STREAMS = 1 << 20
LUXURY = 2048
HBM_COUNT = 1024
FUSED_COUNT = 4096
# Per stream and step: 1024 doubles from a freshly seeded block take 85 refills and stop
# at read position 8; the 4096 fused doubles take the 8 left in that block and then
# 341 refills (advances_for below); 426 LCG advances in all.
IMAD_PER_ADVANCE = 648        # 18 x 18 products of 32 x 32 -> 64 bits = 324 lo + 324 hi
SMS = 152
IMAD_PER_SM_CLK = 64
SM_MAX_MHZ = 2070.0
ALU_PER_SM_CLK = 64
TC_FLOP_PER_ADVANCE = 2 * 80 * 80      # padded 128 x 80 x 80 fp16 product per 128 streams
TC_ALG_FLOP_PER_ADVANCE = 2 * 72 * 72  # the 5,184 byte products of the 72 x 72 folded matrix
CPU_SAMPLE_STREAMS = 16384
SERVE_WARMUP_S = 1.0   # unreported warm-up trace before the serving measurement
# Figures of one ncu capture of the fused tensor kernel (k_fused_tc): DRAM
# bytes (read + write) per stream and launch, and ALU-pipe instructions per refill.
# They describe the kernel as compiled from the sources whose digest is `src_sha`
# (kernel_sources_sha); once those sources change, the figures are reported as null.
TC_FUSED_CAPTURE = {"dram_bytes_per_stream": 76.2, "alu_instr_per_refill": 167, "streams": 262144,
                    "src_sha": "a19c753920aa4dab"}
KERNEL_SOURCES = ("rlxpp_tensor.cu", "rlxpp_arith.cuh", "rlxpp_drawloop.cuh", "rlxpp_state.cuh",
                  "rlxpp_internal.h", "rlxpp_batch.h", "rlxpp_fixmath.cuh", "rlxpp_fixmath_tables.h")


def kernel_sources_sha():
    """Digest of the sources the tensor draw kernels compile from (first 16 hex digits)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_02504_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def tensor_roofline(kernel, advances, ms, peak_tflops, peak_source, n_streams):
    """Roofline of a tensor-path draw kernel: the algorithmic 72 x 72 byte products per
    advance (5,184 multiply-adds, 10,368 flop) over the kernel's CUDA-event time, against
    the measured dense fp16/bf16 tensor peak.  The ALU-pipe view and the DRAM traffic
    come from the recorded ncu capture while the kernel's sources are unchanged."""
    achieved = advances * TC_ALG_FLOP_PER_ADVANCE / (ms * 1e-3) / 1e12
    cap = TC_FUSED_CAPTURE
    current = cap["src_sha"] is not None and cap["src_sha"] == kernel_sources_sha()
    r = {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
         "frac": achieved / peak_tflops, "peak_source": peak_source,
         "work": f"{advances} advances x {TC_ALG_FLOP_PER_ADVANCE} flop (5,184 byte products of A's folded "
                 f"72 x 72 matrix with X's bytes per advance)",
         "padded_mma_tflops": advances * TC_FLOP_PER_ADVANCE / (ms * 1e-3) / 1e12,
         "traffic": cap["dram_bytes_per_stream"] * n_streams if current else None,
         "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel on "
                            f"{cap['streams']} streams, scaled by streams; sources {cap['src_sha']}"
                            if current else "null: no ncu capture of the kernel as currently built")}
    if current and cap["alu_instr_per_refill"]:
        alu = advances * cap["alu_instr_per_refill"] / (ms * 1e-3) / 1e12
        peak_alu = SMS * ALU_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
        r["secondary_alu_pipe"] = {"what": "ALU-pipe instructions issued (ncu count per refill), not "
                                           "algorithmic work", "instr_per_refill": cap["alu_instr_per_refill"],
                                   "achieved_tops": alu, "peak_tops": peak_alu, "frac": alu / peak_alu,
                                   "peak_source": "derived: 152 SMs x 64 ALU lanes/clk x 2070 MHz"}
    return r


def advances_for(count, pos_words, need=2):
    """Refills needed to draw `count` values of `need` words from read position pos."""
    room = max(0, (24 - pos_words) // need)
    head = min(count, room)
    rest = count - head
    per = 24 // need
    adv = -(-rest // per)
    last = rest - (adv - 1) * per if adv else 0
    new_pos = pos_words + head * need if adv == 0 else last * need
    return adv, new_pos


ADV_HBM, POS_AFTER_HBM = advances_for(HBM_COUNT, 0)
ADV_FUSED, _ = advances_for(FUSED_COUNT, POS_AFTER_HBM)
ADV_PER_STREAM = ADV_HBM + ADV_FUSED


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms in the background.  start()
    returns once the first sample is written, so that sampling runs before the timed region
    begins; begin()/end() mark that region, and the reported clock is the median of the
    samples taken inside it (of all samples when the region is too short to hold one)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.path = None
        self.t_begin = self.t_end = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
                 str(self.PERIOD_MS), "-i", self.gpu], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        deadline = time.time() + 3.0
        while time.time() < deadline and self.proc.poll() is None:
            with open(self.path) as fh:
                if fh.read().count("\n") >= 1:
                    break
            time.sleep(0.01)

    def begin(self):
        self.t_begin = datetime.datetime.now()

    def end(self):
        self.t_end = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(2.5 * self.PERIOD_MS / 1000)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def when(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                return None

        inside = [r for r in rows if self.t_begin and self.t_end and when(r) and self.t_begin <= when(r) <= self.t_end]
        use = inside or rows
        sm = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "samples_in_timed_region": len(inside), "period_ms": self.PERIOD_MS}


def cpu_oracle_sample(n_sample, first_seed, threads=None):
    """The oracle as it stands on the host cores: seed n_sample streams (Python big
    integers), then 1024 doubles and 4096 fused doubles per stream (C recurrence,
    one thread per stream range).  Returns (seconds, doubles, threads)."""
    import numpy as np

    from oracle import swb_lib as S
    from tests.oracle_side import StreamSet
    S.build()
    threads = threads or S.default_threads()
    seeds = np.arange(first_seed, first_seed + n_sample, dtype=np.uint64)
    t0 = time.perf_counter()
    ss = StreamSet.from_seeds(seeds, LUXURY)
    S.draw_many(ss.words, ss.carry, ss.pos, LUXURY, HBM_COUNT, S.KIND_F64, threads=threads)
    S.sum_hist_many(ss.words, ss.carry, ss.pos, LUXURY, FUSED_COUNT, threads=threads)
    dt = time.perf_counter() - t0
    return dt, n_sample * (HBM_COUNT + FUSED_COUNT), threads


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values of x (the slowest rank's time); x itself when
    there is one rank.  A collective of the benchmark only, not of the data path."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_doubles_per_s(n_streams_per_rank, world, ms_per_step):
    """Doubles of all ranks per step (each rank draws for its own streams) over the
    slowest rank's time per step."""
    return n_streams_per_rank * (HBM_COUNT + FUSED_COUNT) * world / (ms_per_step * 1e-3)


def workload_config(n_streams, world):
    return {"workload": f"{n_streams} streams x {world} ranks, p={LUXURY}: seed (stream i = seed-1 state "
                        f"skipped by i*2^96 advances) + {HBM_COUNT} f64/stream to HBM + {FUSED_COUNT} "
                        f"f64/stream fused exact sum + 256-bin histogram",
            "streams_per_gpu": n_streams, "luxury": LUXURY, "doubles_per_stream_per_step": HBM_COUNT + FUSED_COUNT,
            "advances_per_stream_per_step": ADV_PER_STREAM, "hbm_bytes_per_step": n_streams * HBM_COUNT * 8,
            "l2": "each step writes 8 GiB (> 129 MB L2); no explicit flush", "parallelism": f"streams x{world}"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_sample = args.cpu_sample
    for _ in range(args.warmup):
        cpu_oracle_sample(min(n_sample, 1024), 1)
    times = []
    threads = None
    doubles = 0
    for _ in range(args.steps):
        dt, doubles, threads = cpu_oracle_sample(n_sample, 1)
        times.append(dt)
    tot = sum(times)
    value = doubles * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(args.streams, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"first {n_sample} of the {args.streams} streams per step: seed + "
                                       f"{HBM_COUNT} f64 + {FUSED_COUNT} fused f64 each (C recurrence oracle, "
                                       f"{threads} threads), {tot / args.steps:.1f} s wall and "
                                       f"{tot / args.steps * threads:.0f} core-seconds per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2106_02504_gb300 as P
    nat = P.native
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    from paper_2106_02504_gb300 import workloads as W
    n = args.streams
    seeds_h = W.rank_seeds(rank, world, n)
    seeds = torch.from_numpy(seeds_h.view(np.int64)).to(dev)
    g = nat.Generator(n, [LUXURY], seeds)
    out = torch.empty((n, HBM_COUNT), dtype=torch.float64, device=dev)
    sums = torch.zeros(n, dtype=torch.int64, device=dev)
    hist = torch.zeros(256, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        nat.rlxpp_seed(g.handle, seeds, sp)
        if ev:
            ev[1].record(stream)
        nat.rlxpp_draw_f64(g.handle, out, HBM_COUNT, None, None, sp)
        if ev:
            ev[2].record(stream)
        nat.rlxpp_draw_f64_sum_hist(g.handle, FUSED_COUNT, sums, hist, sp)
        if ev:
            ev[3].record(stream)

    def barrier():
        if dist is not None:
            dist.barrier()

    def time_path(path):
        g.set_path(path)
        for _ in range(args.warmup):
            step()
        g.sync(sp)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local_rank)
        barrier()
        torch.cuda.synchronize()
        clk.start()
        clk.begin()
        t0.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
        clk.end()
        barrier()
        clocks = clk.stop()
        g.sync(sp)
        ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)
        per_kernel = {
            "seed": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
            "draw_f64_hbm": statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
            "draw_f64_sum_hist": statistics.mean(e[2].elapsed_time(e[3]) for e in evs),
        }
        return ms / args.steps, per_kernel, clocks

    launches_per_step = 3
    # write-only HBM bandwidth on the same 8 GiB buffer (torch's fill kernel), next to
    # the measured copy peak: the HBM kernel only writes
    hbm_write_gbs = n * HBM_COUNT * 8 / (_time_events(lambda: out.zero_(), 3, stream) * 1e-3) / 1e9
    peaks = load_peaks()
    imad_peak = SMS * IMAD_PER_SM_CLK * SM_MAX_MHZ * 1e6  # IMAD ops/s, derived
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    f16_peak = peaks.get("bf16_tflops", 1900.0)  # dense f16 and bf16 run at the same rate
    path_ids = {"imad": nat.RLXPP_PATH_IMAD, "tensor": nat.RLXPP_PATH_TENSOR}
    paths = {}
    for name in args.path.split(","):
        ms_step, per_kernel, clocks = time_path(path_ids[name])
        kern = {}
        for kname, kms in per_kernel.items():
            entry = {"ms": kms, "share": kms / sum(per_kernel.values())}
            adv = {"draw_f64_hbm": n * ADV_HBM, "draw_f64_sum_hist": n * ADV_FUSED}.get(kname)
            if adv:
                entry["advances_per_s"] = adv / (kms * 1e-3)
                entry["imad_equiv_frac"] = adv * IMAD_PER_ADVANCE / (kms * 1e-3) / imad_peak
                if name == "tensor":  # 128 x 80 x 80 fp16 MMA per 128-stream tile and refill
                    entry["tensor_tflops"] = adv * TC_FLOP_PER_ADVANCE / (kms * 1e-3) / 1e12
                    entry["tensor_frac"] = entry["tensor_tflops"] / f16_peak
                    entry["tensor_alg_frac"] = adv * TC_ALG_FLOP_PER_ADVANCE / (kms * 1e-3) / 1e12 / f16_peak
            if kname == "draw_f64_hbm":
                entry["hbm_gbs"] = n * HBM_COUNT * 8 / (kms * 1e-3) / 1e9
                entry["hbm_frac"] = entry["hbm_gbs"] / hbm_peak
                entry["hbm_write_peak_gbs"] = hbm_write_gbs
                entry["hbm_write_frac"] = entry["hbm_gbs"] / hbm_write_gbs
            kern[kname] = entry
        paths[name] = {"ms_per_step": ms_step, "value": whole_job_doubles_per_s(n, world, ms_step),
                       "kernels": kern, "per_kernel_ms": per_kernel, "clocks": clocks}
    best = max(paths, key=lambda k: paths[k]["value"])
    ms_step, per_kernel, clocks = paths[best]["ms_per_step"], paths[best]["per_kernel_ms"], paths[best]["clocks"]
    advances_step = n * ADV_PER_STREAM * world
    value = whole_job_doubles_per_s(n, world, ms_step)
    dom = max(per_kernel, key=per_kernel.get)
    adv = {"draw_f64_sum_hist": n * ADV_FUSED, "draw_f64_hbm": n * ADV_HBM}.get(dom, 0)
    if best == "imad":
        achieved = adv * IMAD_PER_ADVANCE / (per_kernel[dom] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom + " (k_draw, integer pipe)", "achieved": achieved,
                    "peak": imad_peak / 1e12, "unit": "Top/s (32-bit IMAD, 648 per advance)",
                    "frac": achieved / (imad_peak / 1e12),
                    "peak_source": "derived: 152 SMs x 64 IMAD/clk x 2070 MHz", "traffic": None}
    else:
        tc_name = {"draw_f64_sum_hist": "k_fused_tc", "draw_f64_hbm": "k_values_tc<f64>"}.get(dom, "k_seed")
        roofline = tensor_roofline(f"{dom} ({tc_name}, tensor path)", adv, per_kernel[dom], f16_peak,
                                   "MEASURED_PEAKS bf16_tflops (burst; dense fp16 runs at the bf16 rate)", n)
    for name in paths:
        paths[name].pop("per_kernel_ms")
    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "u32", "data": "synthetic",
              "config": dict(workload_config(n, world), path=best),
              "advances_per_s": advances_step / (ms_step * 1e-3),
              "gpu_launches": launches_per_step * args.steps, "kernels": paths[best]["kernels"],
              "roofline": roofline, "clocks": clocks, "paths": paths}
    g.set_path(path_ids[best])

    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        result["e2e"] = run_e2e(args, nat, g, seeds_h, n, world, dev, dist)
    g.close()
    del out
    if not args.only_main and world == 1:  # single-GPU workloads: reported at N = 1
        torch.cuda.empty_cache()
        result["other_workloads"] = {
            "single_stream": bench_single_stream(nat, dev),
            "mixed_batch": bench_mixed_batch(nat, dev, args),
            "skip": bench_skip(nat, dev),
            "normal": bench_normal(nat, dev),
            "exponential": bench_normal(nat, dev, exponential=True),
            "serving": bench_serving(args),
        }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, doubles, threads = cpu_oracle_sample(args.cpu_sample, 1)
        result["cpu_baseline"] = {
            "value": doubles / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {args.cpu_sample} of the {n} streams: seed + {HBM_COUNT} f64 + {FUSED_COUNT} "
                      f"fused f64 each (C recurrence oracle, {threads} threads), {dt:.1f} s wall, "
                      f"{dt * threads:.0f} core-seconds"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def _time_events(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_single_stream(nat, dev):
    """Seed 1, p = 2048, 2^20 doubles from one stream: one thread (serial refills) and
    the same segment split by jump-ahead over many threads (batched requests)."""
    import numpy as np
    import torch
    n = 1 << 20
    st = torch.cuda.current_stream()
    g = nat.Generator(1, [LUXURY], torch.ones(1, dtype=torch.int64, device=dev))
    out = torch.empty(n, dtype=torch.float64, device=dev)
    adv = advances_for(n, 0)[0]
    serial = {}
    for name, pid in (("warp", nat.RLXPP_PATH_WARP), ("tensor", nat.RLXPP_PATH_TENSOR), ("imad", nat.RLXPP_PATH_IMAD)):
        g.set_path(pid)
        ms = _time_events(lambda: nat.rlxpp_draw_f64(g.handle, out, n, None, None, st.cuda_stream), 2, st)
        serial[name] = {"ms": ms, "ns_per_advance": ms * 1e6 / adv}
    best = min(serial, key=lambda k: serial[k]["ms"])
    ms_serial = serial[best]["ms"]
    g.set_path(nat.RLXPP_PATH_TENSOR)
    req = np.zeros(1, dtype=nat.request_dtype())
    req[0] = (0, 0, 0, nat.RLXPP_KIND_F64, n, 0)
    tuning = nat.rlxpp_autotune_requests(g.handle, req, None, out)
    plan = nat.rlxpp_plan_requests(g.handle, req, 0, tuning)
    ms_split = _time_events(lambda: nat.rlxpp_run_plan(g.handle, plan, None, out, st.cuda_stream), 5, st)
    items = nat.rlxpp_plan_items(plan)
    nat.rlxpp_destroy_plan(plan)
    g.close()
    return {"doubles": n, "advances": adv,
            "serial": {"ms": ms_serial, "doubles_per_s": n / (ms_serial * 1e-3),
                       "ns_per_advance": ms_serial * 1e6 / adv, "path": best, "by_path": serial},
            "split": {"ms": ms_split, "doubles_per_s": n / (ms_split * 1e-3), "chunks": items,
                      "tuning": tuning_dict(tuning)}}


def tuning_dict(t):
    """A request tuning (chunk_blocks, blocks_per_sm, path, threads_per_block) for the
    JSON line; threads per block 0 is the default, 128."""
    return {"chunk_blocks": t[0], "blocks_per_sm": t[1], "path": t[2], "threads_per_block": t[3] or 128}


def bench_mixed_batch(nat, dev, args):
    """65,536 streams, luxury uniform over {24, 223, 389, 2048}, counts log-uniform in
    [1, 10^6], u24/f64 50/50: one tuned plan captured in a CUDA graph and replayed,
    against the plain per-stream kernels (one thread per stream) on the same work."""
    import numpy as np
    import torch

    from paper_2106_02504_gb300 import workloads as W
    n = args.batch_streams
    levels, lvl, counts, is_f64 = W.batch_mix(n, seed=3)
    seeds = torch.from_numpy(np.arange(1, n + 1, dtype=np.uint64).view(np.int64)).to(dev)
    g = nat.Generator(n, levels, seeds, torch.from_numpy(lvl).to(dev))
    kind = is_f64.astype(np.uint32)
    offs = np.zeros(n, dtype=np.int64)
    for k in (0, 1):
        idx = np.nonzero(kind == k)[0]
        offs[idx] = np.concatenate([[0], np.cumsum(counts[idx])[:-1]])
    n_u, n_f = int(counts[kind == 0].sum()), int(counts[kind == 1].sum())
    reqs = np.zeros(n, dtype=nat.request_dtype())
    reqs["stream"] = np.arange(n)
    reqs["kind"] = kind
    reqs["count"] = counts
    reqs["offset"] = offs
    out_u = torch.empty(max(n_u, 1), dtype=torch.int32, device=dev)
    out_f = torch.empty(max(n_f, 1), dtype=torch.float64, device=dev)
    refills = sum(advances_for(int(c), 0, 2 if f else 1)[0] for c, f in zip(counts, is_f64))
    st = torch.cuda.current_stream()
    t = time.perf_counter()
    if args.batch_tuning:  # a given tuning instead of the tuner's (to profile a known plan)
        tuned = tuple(int(v) for v in args.batch_tuning.split(","))
        assert len(tuned) == 4, "--batch-tuning needs chunk_blocks,blocks_per_sm,path,threads_per_block"
    else:
        tuned = nat.rlxpp_autotune_requests(g.handle, reqs, out_u, out_f)  # picks the kernel too
    tune_s = time.perf_counter() - t
    by_path = {}
    for name, pid in (("tensor", nat.RLXPP_PATH_TENSOR), ("imad", nat.RLXPP_PATH_IMAD), ("warp", nat.RLXPP_PATH_WARP)):
        tuning = (tuned[0], tuned[1], pid, tuned[3] if pid == tuned[2] else 0)
        t = time.perf_counter()
        plan = nat.rlxpp_plan_requests(g.handle, reqs, 0, tuning)
        plan_s = time.perf_counter() - t
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(st)
        with torch.cuda.stream(side):
            nat.rlxpp_run_plan(g.handle, plan, out_u, out_f, side.cuda_stream)
        st.wait_stream(side)
        with torch.cuda.graph(graph):
            nat.rlxpp_run_plan(g.handle, plan, out_u, out_f)
        ms = _time_events(graph.replay, 3, st)
        by_path[name] = {"ms": ms, "values_per_s": int(counts.sum()) / (ms * 1e-3),
                         "advances_per_s": refills / (ms * 1e-3), "chunks": nat.rlxpp_plan_items(plan),
                         "tuning": tuning_dict(tuning),
                         "plan_s": plan_s, "tuner_choice": pid == tuned[2]}
        nat.rlxpp_destroy_plan(plan)
        del graph
    best = min(by_path, key=lambda k: by_path[k]["ms"])
    ms_graph = by_path[best]["ms"]
    # plain per-stream kernels: u24 streams, then f64 streams (the other kind draws 0)
    cu = torch.from_numpy(np.where(kind == 0, counts, 0)).to(dev)
    cf = torch.from_numpy(np.where(kind == 1, counts, 0)).to(dev)
    o = torch.from_numpy(offs).to(dev)

    def plain():
        nat.rlxpp_draw_u24(g.handle, out_u, 0, cu, o, st.cuda_stream)
        nat.rlxpp_draw_f64(g.handle, out_f, 0, cf, o, st.cuda_stream)
    ms_plain = _time_events(plain, 1, st)
    g.close()
    values = int(counts.sum())
    return {"streams": n, "values": values, "doubles": n_f, "u24": n_u, "advances": int(refills),
            "output_bytes": n_u * 4 + n_f * 8,
            "batched_graph": dict(by_path[best], path=best, tune_s=tune_s,
                                   tuning_source="given" if args.batch_tuning else "tuner"), "batched_graph_by_path": by_path,
            "plain_per_stream": {"ms": ms_plain, "values_per_s": values / (ms_plain * 1e-3),
                                 "advances_per_s": refills / (ms_plain * 1e-3)},
            "speedup_vs_plain": ms_plain / ms_graph}


def bench_skip(nat, dev):
    """2^18 streams (seeds i + 1, p = 2048) skipped by uniform 128-bit distances, then
    48 doubles each."""
    import numpy as np
    import torch

    from paper_2106_02504_gb300 import workloads as W
    n = 1 << 18
    seeds = torch.from_numpy(np.arange(1, n + 1, dtype=np.uint64).view(np.int64)).to(dev)
    g = nat.Generator(n, [LUXURY], seeds)
    dist = torch.from_numpy(W.skip_distances(n, seed=4).view(np.int64)).to(dev)
    out = torch.empty((n, 48), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()
    ms_skip = _time_events(lambda: nat.rlxpp_skip(g.handle, dist, st.cuda_stream), 3, st)
    ms_draw = _time_events(lambda: nat.rlxpp_draw_f64(g.handle, out, 48, None, None, st.cuda_stream), 3, st)
    g.close()
    return {"streams": n, "skip_ms": ms_skip, "skips_per_s": n / (ms_skip * 1e-3),
            "products_per_stream_max": 32, "draw48_ms": ms_draw}


def bench_normal(nat, dev, n=1 << 20, exponential=False):
    """Gaussian doubles (Box-Muller on pairs of the streams' doubles), or exponential
    doubles (inversion, one double each): 2^20 streams (seeds i + 1, p = 2048), 1024
    values each into an 8 GiB device buffer, both paths."""
    import numpy as np
    import torch
    cnt = 1024
    seeds = torch.from_numpy(np.arange(1, n + 1, dtype=np.uint64).view(np.int64)).to(dev)
    g = nat.Generator(n, [LUXURY], seeds)
    out = torch.empty((n, cnt), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()
    res = {"streams": n, "values_per_stream": cnt}
    for name, pid in (("tensor", nat.RLXPP_PATH_TENSOR), ("imad", nat.RLXPP_PATH_IMAD)):
        g.set_path(pid)
        fn = nat.rlxpp_draw_exp_f64 if exponential else nat.rlxpp_draw_normal_f64
        ms = _time_events(lambda: fn(g.handle, out, cnt, None, None, st.cuda_stream), 3, st)
        res[name] = {"ms": ms, "values_per_s": n * cnt / (ms * 1e-3)}
    g.sync()
    g.close()
    del out
    torch.cuda.empty_cache()
    return res


def _host_cpu_times():
    """Seconds of CPU time of the whole machine from /proc/stat: busy (user, nice,
    system, irq, softirq) and steal; None where it is not available."""
    try:
        with open("/proc/stat") as f:
            v = [int(x) for x in f.readline().split()[1:]]
        hz = os.sysconf("SC_CLK_TCK")
        return {"busy": (v[0] + v[1] + v[2] + v[5] + v[6]) / hz, "steal": (v[7] if len(v) > 7 else 0) / hz}
    except (OSError, ValueError, IndexError):
        return None


def bench_serving(args):
    """10^5 resident streams, Poisson arrivals at 2 10^4 requests/s, counts log-uniform in
    [10^2, 10^7], u24/f64 50/50, outputs copied to pinned host memory; the library's
    native serving loop replays the trace (rlxpp_server_run_trace)."""
    import numpy as np

    from paper_2106_02504_gb300 import workloads as W
    from paper_2106_02504_gb300.serve import NativeServer
    n_res, rate = 100_000, 20_000
    n_req = int(rate * args.serve_seconds)
    arr, stream, counts, is_f64 = W.serving_trace(n_req, rate, n_res, seed=5)
    srv = NativeServer(n_res, pool_bytes=args.serve_pool_gib << 30, n_cuda_streams=args.serve_streams,
                       max_batch=args.serve_max_batch)
    # warm-up: a separate one-second trace through the same server first (its first pass
    # over the pool, the CUDA streams and events), so that the measured trace is the
    # steady state; its latencies are not reported
    srv.run_trace(*W.serving_trace(int(rate * SERVE_WARMUP_S), rate, n_res, seed=6))
    host0, cpu0, t0 = _host_cpu_times(), time.process_time(), time.perf_counter()
    lat = srv.run_trace(arr, stream, counts, is_f64)
    host1, cpu1, t1 = _host_cpu_times(), time.process_time(), time.perf_counter()
    loop = srv.stats()
    srv.close()
    ok = lat >= 0
    f64 = np.asarray(is_f64, dtype=bool)
    secs = float((arr[ok] + lat[ok]).max() - arr[ok].min())
    values, doubles = int(counts[ok].sum()), int(counts[ok & f64].sum())
    stats = {"loop": "native (rlxpp_server_run_trace)", "requests": int(ok.sum()), "rejected": int((~ok).sum()),
             "values": values, "doubles": doubles, "seconds": secs, "values_per_s": values / secs,
             "doubles_per_s": doubles / secs, "p50_ms": float(np.percentile(lat[ok], 50) * 1e3),
             "p99_ms": float(np.percentile(lat[ok], 99) * 1e3), "max_ms": float(lat[ok].max() * 1e3)}
    # the loop is one host thread: CPU taken from this machine by others (steal) shows
    # up as latency
    if host0 and host1:
        stats["host"] = {"steal_s": round(host1["steal"] - host0["steal"], 3),
                         "busy_s": round(host1["busy"] - host0["busy"], 3), "cores": os.cpu_count(),
                         "loop_cpu_share": round((cpu1 - cpu0) / (t1 - t0), 3)}
    stats["launch"] = {"max_host_ms": loop["max_launch_us"] / 1e3, "slow_launches": loop["slow_launches"]}
    # where a batch's time went on the device (CUDA events on its stream): the request
    # kernel, and the device-to-host copies after it
    nb = max(loop["batches_timed"], 1)
    stats["device"] = {"batches": loop["batches_timed"], "kernel_ms_mean": loop["kernel_us_sum"] / nb / 1e3,
                       "kernel_ms_max": loop["kernel_us_max"] / 1e3, "copy_ms_mean": loop["copy_us_sum"] / nb / 1e3,
                       "copy_ms_max": loop["copy_us_max"] / 1e3}
    # a backlog that builds up over the trace shows as a higher tail in its second half
    late = ok & (arr >= arr[ok].min() + 0.5 * (arr[ok].max() - arr[ok].min()))
    if late.any():
        stats["p99_second_half_ms"] = float(np.percentile(lat[late], 99) * 1e3)
    stats.update({"resident_streams": n_res, "arrival_rate_hz": rate, "trace_seconds": args.serve_seconds,
                  "warmup_trace_seconds": SERVE_WARMUP_S,
                  "pool_bytes": args.serve_pool_gib << 30, "cuda_streams": args.serve_streams,
                  "max_batch": args.serve_max_batch})
    return stats


def run_e2e(args, nat, g, seeds_h, n, world, dev, dist):
    import numpy as np
    import torch
    seeds_pin = torch.from_numpy(seeds_h.view(np.int64)).pin_memory()
    out_pin = torch.empty((n, HBM_COUNT), dtype=torch.float64).pin_memory()
    sums = torch.zeros(n, dtype=torch.int64, device=dev)
    hist = torch.zeros(256, dtype=torch.int64, device=dev)
    sums_h = torch.empty(n, dtype=torch.int64).pin_memory()
    hist_h = torch.empty(256, dtype=torch.int64).pin_memory()
    sp = torch.cuda.current_stream().cuda_stream

    def step():
        nat.rlxpp_seed(g.handle, seeds_pin, sp)                              # host seeds
        nat.rlxpp_draw_f64_host_async(g.handle, out_pin, HBM_COUNT, sp)       # host output
        nat.rlxpp_draw_f64_sum_hist(g.handle, FUSED_COUNT, sums, hist, sp)   # under its copies
        sums_h.copy_(sums, non_blocking=True)
        hist_h.copy_(hist, non_blocking=True)
        nat.rlxpp_host_wait(g.handle, sp)
        torch.cuda.current_stream().synchronize()

    # the device-to-host link in this run: 1 GiB from device memory into the pinned
    # output, median of three copies (the e2e leg moves 8.6 GB per step through it)
    probe = torch.empty(1 << 27, dtype=torch.float64, device=dev)
    probe.fill_(1.0)
    link = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out_pin.view(-1)[: 1 << 27].copy_(probe, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        link.append((8 << 27) / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del probe
    link_gbs = sorted(link)[1]
    steps = max(1, min(args.steps, 5))
    step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    marks = [t0]
    for _ in range(steps):
        step()
        marks.append(time.perf_counter())
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
    doubles = n * (HBM_COUNT + FUSED_COUNT) * world * steps
    d2h = n * HBM_COUNT * 8 + n * 8 + 256 * 8
    return {"value": doubles / dt, "unit": UNIT, "h2d_bytes_per_step": n * 8,
            "d2h_bytes_per_step": d2h, "steps": steps, "d2h_link_gbs": round(link_gbs, 1),
            "link_frac": round(d2h * steps / dt / 1e9 / link_gbs, 3),
            "step_ms": [round((b - a) * 1e3, 2) for a, b in zip(marks, marks[1:])],
            "how": "rlxpp_seed from pinned host seeds, rlxpp_draw_f64_host_async into pinned host memory "
                   "(library-staged, copied on the library's copy stream while the fused sum/hist draw runs), "
                   "sums+hist read back, rlxpp_host_wait; wall clock"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--streams", type=int, default=N_STREAMS)
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_STREAMS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-main", action="store_true", help="skip the other workloads")
    ap.add_argument("--only-normal", action="store_true",
                    help="run only the Gaussian and exponential workloads on --streams streams (for profiling)")
    ap.add_argument("--only-serve", action="store_true", help="run only the serving trace (for profiling)")
    ap.add_argument("--only-batch", action="store_true",
                    help="run only the mixed batch on --batch-streams streams (for profiling)")
    ap.add_argument("--path", default="imad,tensor", help="refill paths to time; the faster one is reported")
    ap.add_argument("--batch-streams", type=int, default=65536)
    ap.add_argument("--batch-tuning", default="",
                    help="chunk_blocks,blocks_per_sm,path,threads_per_block for the mixed batch instead of "
                         "the tuner's choice (profiling)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-max-batch", type=int, default=512)
    ap.add_argument("--serve-pool-gib", type=int, default=8)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only_batch:
        import torch
        from paper_2106_02504_gb300 import build as _b
        _b.build()
        import paper_2106_02504_gb300._rlxpp as nat
        print(json.dumps({"workload": "mixed_batch", **bench_mixed_batch(nat, torch.device("cuda", local_rank), args)}))
        return 0
    if args.only_serve:
        from paper_2106_02504_gb300 import build as _b
        _b.build()
        print(json.dumps({"workload": "serving", **bench_serving(args)}))
        return 0
    if args.only_normal:
        import torch
        from paper_2106_02504_gb300 import build as _b
        _b.build()
        import paper_2106_02504_gb300._rlxpp as nat
        dev = torch.device("cuda", local_rank)
        print(json.dumps({"workload": "normal", **bench_normal(nat, dev, args.streams)}))
        print(json.dumps({"workload": "exponential", **bench_normal(nat, dev, args.streams, exponential=True)}))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        return run_native(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
