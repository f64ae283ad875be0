#!/usr/bin/env python3
"""Compute-actor benchmark on one GB300 per rank.

Workload (one step): the batched-factorization configuration -- 1024
factorization actors with geometric(mean 64) mailbox lengths (65,162
messages), each message a semiprime p*q with p, q random primes in
[2^24, 2^28).  A step sends every message to its actor's device mailbox,
drains all mailboxes in one persistent launch and writes every reply.

Reported on one JSON line:
  value        msgs/s of the persistent batched path, inputs resident in HBM,
               device time of the K timed steps (CUDA events on the
               runtime's stream); L2 flushed between steps
  latency_ms   p50 / p99 of (reply written - step start), device clock
  per_message_launch   the same workload with one kernel launch per message
  e2e          msgs/s through the host C API (caf_gpu_request_batch +
               caf_gpu_await_batch): messages from pinned host memory,
               replies back to pinned host memory, inside the timed region
  roofline     the drain kernel against the integer-multiply peak
  cpu_baseline the CPU oracle on a bounded sample, host cores
With --impl reference the CPU oracle is the measured program.
Multi-GPU (torchrun): every rank runs its own replica of the workload
(weak scaling, no data-path collective); value = all messages / max time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1505_07368_gb300 import workloads as W  # noqa: E402

METRIC = "compute-actor msgs/sec and p99 latency vs per-message-launch form, same GB300"
UNIT = "msgs/s"
WORKLOAD = ("batched factorization actors: 1024 actors, geometric(mean 64) mailbox lengths, "
            "semiprimes with prime factors in [2^24, 2^28), one persistent launch per step")
L2_FLUSH_BYTES = 256 << 20
IMAD_PER_SM_CLK = 64          # 32-bit integer multiply(-add) lanes per SM per clock
FACTOR_DRAM_BYTES_PER_MSG = (111.944865e9 + 23.120384e6) / 65162   # ncu, the factor drain (see its roofline)
MULS_PER_TEST = 3             # the Montgomery divisibility test: m0, n + m0*p, m1


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--factor-batch", type=int, default=16)
    ap.add_argument("--factor-warps", type=int, default=8)
    ap.add_argument("--ctas-per-sm", type=int, default=2)
    ap.add_argument("--skip-per-message", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--max-messages", type=int, default=None, help="truncate the workload (profiling)")
    ap.add_argument("--workload", choices=["factor", "gemm", "ring", "serve", "mailbox", "small", "mandel", "spawn"],
                    default="factor",
                    help="factor: the batched-factorization line (default); the others measure the "
                         "GEMM, token-ring, serving and mailbox-traffic configurations")
    ap.add_argument("--no-autotune", action="store_true", help="use --factor-batch/--factor-warps as given")
    ap.add_argument("--requests", type=int, default=1_000_000, help="serve: requests in the trace")
    ap.add_argument("--scheduler", choices=["global", "steal"], default="global",
                    help="ready-actor scheduler (factor, ring, mailbox, spawn): one global queue or work stealing")
    ap.add_argument("--factor-split", type=int, default=0,
                    help="factor, ring, serve: split large factor batches over idle teams, up to this many "
                         "segments (0: the runtime's automatic choice, small device batches only; 1: off)")
    ap.add_argument("--gemm-items", type=int, default=None, help="gemm: work items per CTA round (default: the fixed schedule)")
    ap.add_argument("--gemm-tile-n", type=int, default=None, help="gemm: BF16 output tile width, 128 or 256 (default: the fixed schedule)")
    ap.add_argument("--ring-incarnations", type=int, default=4,
                    help="ring: also run the rings re-created this many times on the device (0: skip)")
    ap.add_argument("--fork-n", type=int, default=20, help="spawn: recursion counter n (2^(n+1) - 2 spawns per step)")
    ap.add_argument("--mandel-iters", default="120,1200", help="mandel: maximum iterations to run (comma list)")
    ap.add_argument("--mandel-shapes", default="single,image,row",
                    help="mandel: message shapes to run (single: one image per step; image; row)")
    ap.add_argument("--mandel-images", type=int, default=0,
                    help="mandel: images per step (0: 100 as whole images, 10 as rows)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed plumbing (control plane only)
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None
        self.path = f"/tmp/cafgpu_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def physical_gpu(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# two-sided 95 % quantiles of Student's t distribution, degrees of freedom 1..30
_T975 = (12.706, 4.303, 3.182, 2.776, 2.571, 2.447, 2.365, 2.306, 2.262, 2.228, 2.201, 2.179, 2.160, 2.145,
         2.131, 2.120, 2.110, 2.101, 2.093, 2.086, 2.080, 2.074, 2.069, 2.064, 2.060, 2.056, 2.052, 2.048,
         2.045, 2.042)


def timing_stats(times_s, units_per_step=None):
    """Per-step times (seconds) -> mean, sample standard deviation and the 95 %
    confidence interval of the mean (Student's t), in ms; with units_per_step,
    also the interval of the rate units / mean time."""
    x = np.asarray(times_s, dtype=np.float64) * 1e3
    n = int(x.size)
    out = {"runs": n, "mean_ms": float(x.mean()), "min_ms": float(x.min()), "max_ms": float(x.max())}
    if n >= 2:
        sd = float(x.std(ddof=1))
        hw = (_T975[n - 2] if n - 1 <= len(_T975) else 1.96) * sd / np.sqrt(n)
        out.update({"std_ms": sd, "ci95_ms": [out["mean_ms"] - hw, out["mean_ms"] + hw], "ci95_halfwidth_ms": hw})
        if units_per_step is not None and out["mean_ms"] - hw > 0:
            out["rate_ci95"] = [units_per_step / ((out["mean_ms"] + hw) * 1e-3),
                                units_per_step / ((out["mean_ms"] - hw) * 1e-3)]
    return out


# ---------------------------------------------------------------------------
# algorithmic work: odd primes up to each message's smallest factor
# ---------------------------------------------------------------------------
def odd_prime_counts(p: np.ndarray) -> np.ndarray:
    """Number of odd primes <= p for each p (host sieve of the odd numbers)."""
    limit = int(p.max())
    half = limit // 2 + 1                      # index i stands for 2i + 1
    comp = np.zeros(half, dtype=bool)
    comp[0] = True
    r = int(limit ** 0.5) + 1
    for i in range(1, r // 2 + 1):
        if not comp[i]:
            q = 2 * i + 1
            comp[(q * q) // 2::q] = True
    odd_primes = 2 * np.nonzero(~comp)[0].astype(np.int64) + 1
    return np.searchsorted(odd_primes, p.astype(np.int64), side="right")


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def cpu_oracle_rate(wl, seconds: float, start: int = 0):
    import oracle
    oracle.build()
    done = 0
    t0 = time.perf_counter()
    i = start
    while True:
        oracle.factor_batch(wl.n[i:i + 1])
        done += 1
        i = (i + 1) % wl.count
        el = time.perf_counter() - t0
        if el >= seconds and done >= 2:
            break
    return done / el, done, el


def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return 0
    wl = W.config2()
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, 0.2)
    total_msgs, total_s = 0, 0.0
    for k in range(args.steps):
        rate, done, el = cpu_oracle_rate(wl, per_step, start=k * 7)
        total_msgs += done
        total_s += el
    value = total_msgs / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "messages": wl.count},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{total_msgs} messages of the workload, single-threaded trial division"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1505_07368_gb300 import cafgpu as C

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local_rank)

    wl = W.config2(max_messages=args.max_messages)
    count = wl.count
    tuned = None
    if not args.no_autotune:
        from paper_1505_07368_gb300 import autotune
        best, table = autotune.tune_factor(wl.actor, wl.n, wl.n_actors, (1 << 56) - 1,
                                           runtime_kwargs={"mailbox_capacity": 512},
                                           log=lambda m: print(m, file=sys.stderr))
        args.factor_batch, args.factor_warps, args.ctas_per_sm = (best["factor_batch"], best["factor_warps"],
                                                                  best["ctas_per_sm"])
        tuned = {"best": best, "measured": [[c, round(t * 1e3, 2)] for c, t in table] or "cached"}
    rt = C.Runtime(max_factor_n=(1 << 56) - 1, max_actors=wl.n_actors, mailbox_capacity=512,
                   ingress_capacity=1 << 17, max_inflight_requests=1 << 17, factor_batch=args.factor_batch,
                   factor_warps=args.factor_warps, ctas_per_sm=args.ctas_per_sm, scheduler=_sched(args),
                   factor_split=args.factor_split)
    for _ in range(wl.n_actors):
        rt.spawn(C.FACTOR_U64)
    m = np.zeros(count, C.DMSG_DTYPE)
    m["actor"] = wl.actor
    m["kind"] = C.FACTOR_U64
    m["u64"] = wl.n
    m["sender"] = wl.sender
    m["sender_seq"] = wl.sender_seq
    m["tag"] = np.arange(count)
    d_msgs = torch.from_numpy(m.view(np.uint8).copy()).to(dev)
    d_rep = torch.zeros(count * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.ExternalStream(rt.stream(), device=dev)
    torch.cuda.synchronize()

    def step():
        rt.mark()
        rt.request_batch_device(d_msgs.data_ptr(), count, d_rep.data_ptr())

    def check(rep):
        ok = (np.all(rep["status"] == 0) and np.array_equal(rep["r0"], wl.p) and np.array_equal(rep["r1"], wl.q))
        if not ok:
            raise SystemExit("bench: replies differ from the workload's factors")

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        step()
        rt.stream_sync()
    check(d_rep.cpu().numpy().view(C.DREPLY_DTYPE))
    rt.stats()  # reset counters

    sampler = ClockSampler(physical_gpu(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    rt.stream_sync()
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    st = rt.stats()
    rep = d_rep.cpu().numpy().view(C.DREPLY_DTYPE).copy()
    check(rep)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_s = sum(step_ms) / 1e3
    t_mark = st["t_mark"]
    lat_ms = (rep["t_done"].astype(np.int64) - np.int64(t_mark)) / 1e6
    dev_s_max = allreduce_max(dev_s, world, dev)
    msgs_all = allreduce_sum(float(count * args.steps), world, dev)
    value = msgs_all / dev_s_max

    # roofline: the drain kernel against the integer-multiply peak
    tests_alg = float(odd_prime_counts(wl.p).sum())
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tops = sm_count * IMAD_PER_SM_CLK * sm_max * 1e6 / 1e12
    achieved_tops = MULS_PER_TEST * tests_alg / (dev_s / args.steps) / 1e12
    # DRAM traffic per launch: the drain's dram__bytes_read.sum + dram__bytes_write.sum from one
    # ncu capture (one-pass counters) of this workload's full launch with the current sweep (K=16,
    # W=8, 2 CTAs/SM), per message, times this step's messages.  Other settings: not captured
    # (null).
    traffic = None
    if (args.factor_batch, args.factor_warps, args.ctas_per_sm, args.factor_split) == (16, 8, 2, 0):
        traffic = FACTOR_DRAM_BYTES_PER_MSG * count
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tmul/s",
                "frac": achieved_tops / peak_tops, "traffic": traffic,
                "traffic_basis": "bytes per launch: ncu capture of the full 65,162-message launch, per message" if traffic else None,
                "kernel": "k_drain", "algorithmic_tests_per_step": tests_alg,
                "executed_tests_per_step": st["prime_tests"] / args.steps,
                "peak_basis": f"{sm_count} SMs (device attribute) x {IMAD_PER_SM_CLK} IMAD/clk x {sm_max:.0f} MHz (sm_max_mhz of measured)"}
    # what the test's own instruction mix can reach on this GPU (measured after
    # the timed steps): its high multiply runs at a lower rate than the low one
    rates = C.measure_mul_rates()
    chain = rates["test_chain_mul_per_s"] / 1e12
    roofline["measured_ceiling"] = {
        "unit": "Tmul/s", "test_chain": chain, "mul_lo": rates["mul_lo_per_s"] / 1e12,
        "mul_hi": rates["mul_hi_per_s"] / 1e12, "frac_of_test_chain": achieved_tops / chain,
        "basis": "caf_gpu_measure_mul_rates: 8 independent chains per thread, 8 CTAs x 256 threads per SM"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "messages": count, "actors": wl.n_actors,
                   "factor_batch": args.factor_batch, "factor_warps": args.factor_warps,
                   "ctas_per_sm": args.ctas_per_sm, "scheduler": args.scheduler, "factor_split": args.factor_split,
                   "l2": "flushed between steps (256 MiB write)",
                   "timing": "CUDA events on the runtime stream, per step",
                   "autotune": tuned if tuned else "off"},
        "timing_stats": timing_stats(np.asarray(step_ms) / 1e3, units_per_step=float(count)),
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "max": float(lat_ms.max()), "from": "step start (device clock) to reply written"},
        "gpu_launches": st["launches"],
        "wall_s": wall,
        "roofline": roofline,
        "clocks": clocks,
    }

    # per-message-launch form (same workload, one kernel launch per message)
    if not args.skip_per_message:
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        msgs = (C.Msg * count)()
        for i in range(count):
            msgs[i] = C.Runtime.msg(C.FACTOR_U64, int(wl.n[i]), sender=int(wl.sender[i]), tag=i)
        actors = (wl.actor.astype(np.uint64) + 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        rt.stats()
        e0.record(stream)
        rt.mark()
        h = rt.request_batch(actors, msgs)
        e1.record(stream)
        rrep = rt.await_batch(h, timeout_ns=AWAIT_NS)
        torch.cuda.synchronize()
        pm_s = e0.elapsed_time(e1) / 1e3
        pst = rt.stats()
        if not (np.array_equal(rrep["r0"], wl.p) and np.array_equal(rrep["r1"], wl.q)):
            raise SystemExit("bench: per-message-launch replies differ")
        plat = (rrep["t_done"].astype(np.int64) - np.int64(pst["t_mark"])) / 1e6
        line["per_message_launch"] = {"value": count / pm_s, "unit": UNIT, "launches": pst["launches"],
                                      "p50_ms": float(np.percentile(plat, 50)),
                                      "p99_ms": float(np.percentile(plat, 99)),
                                      "speedup_persistent": value / (count / pm_s)}
        rt.set_backend(C.BACKEND_PERSISTENT)

    # e2e through the host API, host buffers in and out
    if not args.skip_e2e:
        msgs = (C.Msg * count)()
        for i in range(count):
            msgs[i] = C.Runtime.msg(C.FACTOR_U64, int(wl.n[i]), sender=int(wl.sender[i]), tag=i)
        actors = (wl.actor.astype(np.uint64) + 1)
        h = rt.request_batch(actors, msgs)      # warm-up pass
        rt.await_batch(h, timeout_ns=AWAIT_NS)
        rt.sync()
        times = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = rt.request_batch(actors, msgs)
            erep = rt.await_batch(h, timeout_ns=AWAIT_NS)
            times.append(time.perf_counter() - t0)
            rt.sync()
        if not (np.array_equal(erep["r0"], wl.p) and np.array_equal(erep["r1"], wl.q)):
            raise SystemExit("bench: e2e replies differ")
        e2e_s = allreduce_max(float(np.mean(times)), world, dev)
        line["e2e"] = {"value": allreduce_sum(float(count), world, dev) / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": count * 64, "d2h_bytes_per_step": count * 32,
                       "path": "caf_gpu_request_batch + caf_gpu_await_batch (pinned ingress ring, pinned replies)"}

    rt.close()

    if rank == 0:
        rate, done, el = cpu_oracle_rate(wl, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{done} messages of the workload in {el:.1f} s, single-threaded trial division"}
        line["speedup_vs_cpu_oracle"] = value / rate
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# other configurations (measurement lines for the record; the default line is
# the default batched-factorization workload)
# ---------------------------------------------------------------------------
def _sched(args) -> int:
    return 1 if getattr(args, "scheduler", "global") == "steal" else 0


def _note(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


AWAIT_NS = 300_000_000_000     # host waits in the bench give up after 5 minutes


def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


GEMM_SCHEDULE = {"bf16": {"gemm_items_per_round": 8, "gemm_tile_n": 256},
                 "split_bf16x3": {"gemm_items_per_round": 4}}


def run_gemm(args):
    """GEMM actors: 256 actors, 4096 messages, n uniform in {64, ..., 1024}, N(0,1)
    operands (views into a 256 MiB pool), BF16 and split-BF16x3, one drain per step."""
    import torch

    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    wl = W.config3(pool_elems=1 << 26, n_messages=args.max_messages or 4096)
    pool = torch.from_numpy(W.gemm_pool(wl.pool_seed, wl.pool_elems)).cuda()
    sizes = wl.size.astype(np.int64)
    outs = torch.empty(int((4 * sizes * sizes).sum() // 4), dtype=torch.float32, device="cuda")
    c_off = np.concatenate([[0], np.cumsum(sizes * sizes)[:-1]])
    desc = np.zeros(wl.count, C.GEMM_DESC_DTYPE)
    desc["A"] = pool.data_ptr() + 4 * wl.a_off.astype(np.uint64)
    desc["B"] = pool.data_ptr() + 4 * wl.b_off.astype(np.uint64)
    desc["C"] = outs.data_ptr() + 4 * c_off.astype(np.uint64)
    desc["n"] = sizes
    d_desc = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    useful_flops = float((2 * sizes.astype(np.float64) ** 3).sum())
    alg_bytes = float((12 * sizes.astype(np.float64) ** 2).sum())
    peaks = measured_peaks()
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "bf16 operands, f32 accumulate", "data": "synthetic",
            "config": {"workload": f"GEMM actors: 256 actors, {wl.count} messages, n uniform in {{64,...,1024}}, N(0,1)",
                       "messages": wl.count, "l2": "flushed between steps (256 MiB write)"}, "variants": {}}
    for kind, name in ((C.GEMM_BF16, "bf16"), (C.GEMM_SPLIT_BF16X3, "split_bf16x3")):
        # fixed schedules: the fastest of items 2/4/8 (x tile width 128/256
        # for BF16) measured on GB300, one runtime per variant; the GEMM
        # autotuner's GPU timing (a runtime per candidate) stays off
        sched = dict(GEMM_SCHEDULE[name])
        if args.gemm_items is not None:
            sched["gemm_items_per_round"] = args.gemm_items
        if args.gemm_tile_n is not None:
            sched["gemm_tile_n"] = args.gemm_tile_n
        line["config"].setdefault("schedule", {})[name] = dict(sched)
        _note(f"gemm {name}: persistent {sched}")
        with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=wl.n_actors, mailbox_capacity=64, **sched) as rt:
            for _ in range(wl.n_actors):
                rt.spawn(kind)
            m = np.zeros(wl.count, C.DMSG_DTYPE)
            m["actor"] = wl.actor
            m["kind"] = kind
            m["u64"] = d_desc.data_ptr() + np.arange(wl.count, dtype=np.uint64) * 32
            m["tag"] = np.arange(wl.count)
            d_m = torch.from_numpy(m.view(np.uint8).copy()).cuda()
            d_r = torch.zeros(wl.count * 32, dtype=torch.uint8, device="cuda")
            stream = torch.cuda.ExternalStream(rt.stream())
            torch.cuda.synchronize()
            for _ in range(args.warmup):
                rt.request_batch_device(d_m.data_ptr(), wl.count, d_r.data_ptr())
            rt.stream_sync()
            times = []
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.add_(1.0)
                e0, e1 = _events(stream)
                e0.record(stream)
                rt.mark()
                rt.request_batch_device(d_m.data_ptr(), wl.count, d_r.data_ptr())
                e1.record(stream)
                rt.stream_sync()
                times.append(e0.elapsed_time(e1) / 1e3)
            st = rt.stats()
            rep = d_r.cpu().numpy().view(C.DREPLY_DTYPE)
            if not (np.all(rep["status"] == 0) and np.array_equal(rep["r1"], sizes.astype(np.uint64))):
                raise SystemExit("bench: GEMM replies incomplete")
            lat = (rep["t_done"].astype(np.int64) - np.int64(st["t_mark"])) / 1e6
            t = float(np.mean(times))
            mult = 3.0 if kind == C.GEMM_SPLIT_BF16X3 else 1.0
            v = {"value": wl.count / t, "ms_per_step": 1e3 * t, "timing_stats": timing_stats(times, wl.count),
                 "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                 "roofline": {
                     "hbm": {"achieved": alg_bytes / t / 1e9, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                             "frac": alg_bytes / t / 1e9 / peaks.get("hbm_gbs", 6800.0)},
                     "tensor": {"achieved": mult * useful_flops / t / 1e12,
                                "peak": peaks.get("bf16_tflops", 1900.0), "unit": "TFLOP/s",
                                "frac": mult * useful_flops / t / 1e12 / peaks.get("bf16_tflops", 1900.0),
                                "note": "executed flops (split: 3 products per useful one)"}},
                 "useful_tflops": useful_flops / t / 1e12, "gpu_launches": st["launches"]}
            if not args.skip_per_message:
                _note(f"gemm {name}: per-message launch")
                rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
                msgs = (C.Msg * wl.count)()
                for i in range(wl.count):
                    msgs[i] = C.Runtime.msg(kind, n=int(sizes[i]), A=int(desc["A"][i]), B=int(desc["B"][i]),
                                            C=int(desc["C"][i]), tag=i)
                e0, e1 = _events(stream)
                torch.cuda.synchronize()
                e0.record(stream)
                h = rt.request_batch(wl.actor.astype(np.uint64) + 1, msgs)
                e1.record(stream)
                rt.await_batch(h, timeout_ns=AWAIT_NS)
                torch.cuda.synchronize()
                pm = e0.elapsed_time(e1) / 1e3
                v["per_message_launch"] = {"value": wl.count / pm, "ms": 1e3 * pm,
                                           "speedup_persistent": (wl.count / t) / (wl.count / pm)}
            line["variants"][name] = v
    line["value"] = line["variants"]["split_bf16x3"]["value"]
    print(json.dumps(line))
    return 0


def run_ring(args):
    """Mixed workload: 64 rings of 128 actors, token 1000 decremented per hop,
    each master sending 8 factorization requests (factors in [2^30, 2^31)) to its
    ring's worker; the whole workload is one captured CUDA graph per step."""
    import torch

    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    wl = W.config4()
    R, L, rounds = wl.n_rings, wl.ring_len, wl.n.shape[1]
    out = {}
    for label, with_factor in (("tokens_only", False), ("mixed", True)):
        with C.Runtime(max_actors=R * (L + 1), scheduler=_sched(args), factor_split=args.factor_split) as rt:
            d_n = torch.from_numpy(wl.n.astype(np.uint64).reshape(-1).copy()).cuda()
            d_rep = torch.zeros(R * rounds * 32, dtype=torch.uint8, device="cuda")
            masters = []
            for r in range(R):
                worker = rt.spawn(C.FACTOR_U64, mailbox_capacity=16)
                base = worker + 1
                for i in range(L):
                    nxt = base + (i + 1) % L
                    if i == 0:
                        h = rt.spawn(C.RING_TOKEN, mailbox_capacity=4, next=nxt, flags=C.ACTOR_MASTER, worker=worker,
                                     factor_n=d_n.data_ptr() + r * rounds * 8, factor_count=rounds if with_factor else 0,
                                     factor_replies=d_rep.data_ptr() + r * rounds * 32)
                        masters.append(h)
                    else:
                        rt.spawn(C.RING_TOKEN, mailbox_capacity=4, next=nxt)
            m = np.zeros(R, C.DMSG_DTYPE)
            m["actor"] = np.array(masters, np.uint32) - 1
            m["kind"] = C.RING_TOKEN | (C.MSG_START << 16)
            m["u64"] = wl.token
            d_m = torch.from_numpy(m.view(np.uint8).copy()).cuda()
            d_r = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            rt.graph_begin()
            rt.reset_actors()
            rt.request_batch_device(d_m.data_ptr(), R, d_r.data_ptr())
            g = rt.graph_end()
            stream = torch.cuda.ExternalStream(rt.stream())
            for _ in range(args.warmup):
                rt.graph_launch(g)
            rt.stream_sync()
            times = []
            for _ in range(args.steps):
                e0, e1 = _events(stream)
                e0.record(stream)
                rt.graph_launch(g)
                e1.record(stream)
                rt.stream_sync()
                times.append(e0.elapsed_time(e1) / 1e3)
            rt.graph_destroy(g)
            t = float(np.mean(times))
            hops = L + wl.token            # deliveries per ring (the 0 travels once around)
            msgs = R * (hops + 1) + (R * rounds if with_factor else 0)
            out[label] = {"ms_per_step": 1e3 * t, "timing_stats": timing_stats(times, msgs),
                          "msgs_per_s": msgs / t, "ns_per_hop": 1e9 * t / hops,
                          "messages": msgs}
            if not args.skip_per_message:
                # the same workload with one kernel launch per message: the host sends
                # each master its start message and launches the messages each wave
                # produces until none is left (one run; it takes seconds)
                rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
                rt.reset_actors()
                d_rep.zero_()
                rt.stream_sync()
                torch.cuda.synchronize()
                rt.stats()                 # restart the launch count
                t0 = time.perf_counter()
                for mst in masters:
                    rt.send(mst, C.Runtime.msg(C.RING_TOKEN, wl.token, flags=C.MSG_START))
                rt.sync()
                tp = time.perf_counter() - t0
                launches = rt.stats()["launches"]
                if with_factor:
                    rep_ = d_rep.cpu().numpy().view(C.DREPLY_DTYPE).reshape(R, rounds)
                    n_ = wl.n.astype(np.uint64)
                    if not (np.all(rep_["status"] == 0) and np.array_equal(rep_["r0"] * rep_["r1"], n_)):
                        raise SystemExit("bench: ring: per-message factor replies wrong")
                out[label]["per_message_launch"] = {"ms": 1e3 * tp, "msgs_per_s": msgs / tp, "launches": launches,
                                                    "speedup_persistent": tp / t,
                                                    "timing": "host wall clock around the sends and caf_gpu_sync"}
    if args.ring_incarnations > 0:
        out["recreated"] = _ring_recreated(args, wl, C)
    lat = C.measure_latency()
    for v in out.values():
        v["hop_in_handoffs"] = v["ns_per_hop"] / lat["handoff_ns"]
        v["hop_in_l2_round_trips"] = v["ns_per_hop"] / lat["load_acquire_ns"]
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": "token rings (64 x 128, token 1000) + "
                      "8 factorization requests per ring, captured CUDA graph", "steps": args.steps,
                      "factor_split": args.factor_split, "latency_probe_ns": lat,
                      "results": out, "value": out["mixed"]["msgs_per_s"]}))
    return 0


def _ring_recreated(args, wl, C):
    """The mixed workload with every ring re-created on the device: each master
    spawns its 127 members from the device actor pool, runs the ring, and
    spawns the next incarnation once all have terminated, args.ring_incarnations
    times; 8 factorization requests per incarnation.  One CUDA graph per step."""
    import torch
    R, L, I = wl.n_rings, wl.ring_len, args.ring_incarnations
    rounds = wl.n.shape[1]
    big = W.config4(n_rings=R * I)
    n = big.n.reshape(R, rounds * I)
    with C.Runtime(max_actors=2 * R, scheduler=_sched(args), factor_split=args.factor_split,
                   fork_pool=R * (L - 1)) as rt:
        d_n = torch.from_numpy(n.astype(np.uint64).reshape(-1).copy()).cuda()
        d_rep = torch.zeros(R * rounds * I * 32, dtype=torch.uint8, device="cuda")
        masters = []
        for r in range(R):
            worker = rt.spawn(C.FACTOR_U64, mailbox_capacity=16)
            masters.append(rt.spawn(C.RING_TOKEN, mailbox_capacity=4, flags=C.ACTOR_MASTER | C.ACTOR_RECREATE,
                                    worker=worker, factor_n=d_n.data_ptr() + r * rounds * I * 8,
                                    factor_count=rounds * I,
                                    factor_replies=d_rep.data_ptr() + r * rounds * I * 32, ring_len=L, incarnations=I))
        m = np.zeros(R, C.DMSG_DTYPE)
        m["actor"] = np.array(masters, np.uint32) - 1
        m["kind"] = C.RING_TOKEN | (C.MSG_START << 16)
        m["u64"] = wl.token
        d_m = torch.from_numpy(m.view(np.uint8).copy()).cuda()
        d_r = torch.zeros(R * 32, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        rt.graph_begin()
        rt.reset_actors()
        rt.request_batch_device(d_m.data_ptr(), R, d_r.data_ptr())
        g = rt.graph_end()
        stream = torch.cuda.ExternalStream(rt.stream())
        for _ in range(args.warmup):
            rt.graph_launch(g)
        rt.stream_sync()
        rt.stats()
        times = []
        for _ in range(args.steps):
            e0, e1 = _events(stream)
            e0.record(stream)
            rt.graph_launch(g)
            e1.record(stream)
            rt.stream_sync()
            times.append(e0.elapsed_time(e1) / 1e3)
        st = rt.stats()
        rt.graph_destroy(g)
        rep_ = d_rep.cpu().numpy().view(C.DREPLY_DTYPE).reshape(R, rounds * I)
        if not (np.all(rep_["status"] == 0) and np.array_equal(rep_["r0"] * rep_["r1"], n.astype(np.uint64))):
            raise SystemExit("bench: ring recreated: factor replies wrong")
        if st["device_spawns"] != args.steps * R * (L - 1) * I:
            raise SystemExit(f"bench: ring recreated: spawned {st['device_spawns']}")
    t = float(np.mean(times))
    hops = (L + wl.token) * I
    msgs = R * (hops + 1 + I) + R * rounds * I        # tokens, START, end-of-incarnation notices, factors
    return {"ms_per_step": 1e3 * t, "timing_stats": timing_stats(times, msgs), "msgs_per_s": msgs / t,
            "ns_per_hop": 1e9 * t / hops, "messages": msgs, "incarnations": I,
            "device_spawns_per_step": R * (L - 1) * I, "spawns_per_s": R * (L - 1) * I / t}


def run_serve(args):
    """Serving: open-loop Poisson arrivals, 70 % factorization (log-uniform factors in
    [2^16, 2^31)), 30 % split-BF16x3 GEMM (n log-uniform in [32, 2048]), 8 GB budget.
    Closed-loop capacity first, then open loop at 0.8 of it, persistent vs per-message."""
    import torch

    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    count = args.requests
    n_f, n_g = 2048, 1024
    pool_elems = 1 << 28            # 1 GiB of operands: larger than L2, so the GEMMs read HBM
    _note(f"serve: drawing the {count}-request trace and a {pool_elems * 4 >> 20} MiB operand pool")
    base_wl = W.config5(n_requests=count, rate=1e6, pool_elems=pool_elems)
    pool_np = W.gemm_pool(base_wl.pool_seed, base_wl.pool_elems)
    pool = torch.from_numpy(pool_np).cuda()
    arena_bytes = 4 << 30
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    result = {"metric": METRIC, "unit": UNIT, "requests": count,
              "workload": "serving: Poisson arrivals, 70% factor / 30% split GEMM, 8 GB budget",
              "operand_pool_bytes": pool_elems * 4, "checks": {}}

    def check(res, wl, label):
        """Every reply: status, factors against the generator's primes, GEMM size;
        split-GEMM error on a seeded sample of the results still intact in the
        arena (a later result may reuse an earlier one's bytes), large n included."""
        isf = wl.kind == C.FACTOR_U64
        bad = int(np.count_nonzero(res["status"] != 0))
        fi = np.nonzero(isf)[0]
        gi = np.nonzero(~isf)[0]
        bad_f = int(np.count_nonzero((res["r0"][fi] != wl.p[fi]) | (res["r1"][fi] != wl.q[fi])))
        bad_g = int(np.count_nonzero(res["r1"][gi] != wl.size[gi].astype(np.uint64)))
        page = 1 << 12
        taken = np.zeros(arena_bytes // page + 1, dtype=bool)
        intact_big, intact = [], []
        for i in gi[::-1]:
            n = int(wl.size[i])
            lo = int(res["c_offset"][i]) // page
            hi = (int(res["c_offset"][i]) + 4 * n * n - 1) // page + 1
            if not taken[lo:hi].any():
                (intact_big if n > 1024 else intact).append(i)
            taken[lo:hi] = True
            if len(intact_big) >= 6 and len(intact) >= 400:
                break
        rng = np.random.default_rng(1505_07368)
        sample = intact_big[:6] + list(rng.choice(intact, size=min(18, len(intact)), replace=False))
        worst = 0.0
        for i in sample:
            n = int(wl.size[i])
            rows = np.unique(rng.integers(0, n, size=24))
            off = int(res["c_offset"][i])
            got = arena[off:off + 4 * n * n].view(torch.float32).view(n, n)[torch.from_numpy(rows).cuda()]
            got = got.cpu().numpy().astype(np.float64)
            A = pool_np[wl.a_off[i]:wl.a_off[i] + n * n].reshape(n, n)
            B = pool_np[wl.b_off[i]:wl.b_off[i] + n * n].reshape(n, n)
            want = A[rows].astype(np.float64) @ B.astype(np.float64)
            err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
            worst = max(worst, err)
        result["checks"][label] = {
            "replies": int(res.size), "bad_status": bad, "bad_factors": bad_f, "factor_replies": int(fi.size),
            "bad_gemm_replies": bad_g, "gemm_replies": int(gi.size),
            "gemm_error_sample": {"messages": len(sample), "large_n": len(intact_big[:6]),
                                  "sizes": sorted(int(wl.size[i]) for i in sample),
                                  "worst_rel_frobenius": worst, "bound": 1e-5,
                                  "reference": "float64 numpy product of the float32 operands, 24 sampled rows"}}
        if bad or bad_f or bad_g or worst > 1e-5 or not intact_big:
            print(json.dumps(result["checks"][label]), file=sys.stderr)
            raise SystemExit(f"bench: serve {label}: replies fail the check")

    def trace(wl, actors_f, actors_g):
        reqs = np.zeros(wl.count, C.SERVE_REQ_DTYPE)
        isf = wl.kind == C.FACTOR_U64
        reqs["actor"] = np.where(isf, np.array(actors_f, np.uint64)[wl.actor % n_f],
                                 np.array(actors_g, np.uint64)[(wl.actor - n_f) % n_g])
        reqs["t_arrival"] = wl.t
        reqs["u64"] = wl.n
        reqs["n"] = wl.size
        reqs["A"] = np.where(isf, 0, pool.data_ptr() + 4 * wl.a_off.astype(np.uint64))
        reqs["B"] = np.where(isf, 0, pool.data_ptr() + 4 * wl.b_off.astype(np.uint64))
        return reqs

    with C.Runtime(max_actors=n_f + n_g, mailbox_capacity=256, max_inflight_requests=1 << 17,
                   ingress_capacity=1 << 17, factor_split=args.factor_split) as rt:
        af = [rt.spawn(C.FACTOR_U64) for _ in range(n_f)]
        ag = [rt.spawn(C.GEMM_SPLIT_BF16X3) for _ in range(n_g)]
        closed = trace(base_wl, af, ag)
        closed["t_arrival"] = 0.0
        torch.cuda.synchronize()
        _note("serve: closed loop")
        res, st = rt.serve_run(closed, arena.data_ptr(), arena_bytes, mem_budget_bytes=8 << 30)
        torch.cuda.synchronize()
        check(res, base_wl, "closed_loop")
        capacity = count / st["wall_s"]
        result["closed_loop"] = {"msgs_per_s": capacity, "wall_s": st["wall_s"]}
        lam = 0.8 * capacity
        wl = W.config5(n_requests=count, rate=lam, pool_elems=pool_elems)
        reqs = trace(wl, af, ag)
        for backend, label in ((C.BACKEND_PERSISTENT, "persistent"), (C.BACKEND_PER_MESSAGE_LAUNCH, "per_message_launch")):
            _note(f"serve: open loop, {label}")
            rt.set_backend(backend)
            res, st = rt.serve_run(reqs, arena.data_ptr(), arena_bytes, mem_budget_bytes=8 << 30)
            torch.cuda.synchronize()
            check(res, wl, label)
            lat = (res["t_done"] - wl.t) * 1e3
            result[label] = {"rate_offered": lam, "msgs_per_s": count / st["wall_s"],
                             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "peak_inflight_bytes": st["peak_inflight_bytes"], "launches": st["launches"]}
    result["value"] = result["persistent"]["msgs_per_s"]
    print(json.dumps(result))
    return 0


def run_small(args):
    """The plain small case (config 1): 1 actor, 1 mailbox, 256 semiprimes with
    prime factors in [2^16, 2^20); the per-message-launch form (the config's
    own method) against the persistent drain, and the oracle on one core."""
    import torch

    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    wl = W.config1()
    out = {}
    for backend, label in ((C.BACKEND_PER_MESSAGE_LAUNCH, "per_message_launch"), (C.BACKEND_PERSISTENT, "persistent")):
        with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=1) as rt:
            a = rt.spawn(C.FACTOR_U64)
            rt.set_backend(backend)
            msgs = (C.Msg * wl.count)()
            for i in range(wl.count):
                msgs[i] = C.Runtime.msg(C.FACTOR_U64, u64=int(wl.n[i]), tag=i)
            actors = np.full(wl.count, a, np.uint64)
            for _ in range(args.warmup):
                rt.await_batch(rt.request_batch(actors, msgs), timeout_ns=AWAIT_NS)
            times, lat = [], []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                h = rt.request_batch(actors, msgs)
                rep = rt.await_batch(h, timeout_ns=AWAIT_NS)
                times.append(time.perf_counter() - t0)
            if not (np.array_equal(rep["r0"], np.minimum(wl.p, wl.q)) and np.array_equal(rep["r1"], np.maximum(wl.p, wl.q))):
                raise SystemExit(f"bench: small {label}: wrong factors")
            t = float(np.mean(times))
            out[label] = {"msgs_per_s": wl.count / t, "ms_per_step": 1e3 * t,
                          "timing_stats": timing_stats(times, wl.count),
                          "launches_per_step": rt.stats()["launches"] / (args.warmup + args.steps)}
    rate, done, secs = cpu_oracle_rate(wl, args.cpu_seconds)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": "plain small case: 1 actor, 1 mailbox, 256 "
                      "semiprimes, prime factors in [2^16, 2^20)", "steps": args.steps,
                      "timing": "host wall clock around request_batch + await_batch (host API, end to end)",
                      "results": out, "value": out["persistent"]["msgs_per_s"],
                      "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"{done} messages in {secs:.1f} s, single-threaded trial division"}}))
    return 0


def run_mailbox(args):
    """Mailbox traffic: SOURCE actors stream into SINK actors (trivial payload),
    N:1 -- 100 sources into one sink, the paper's mailbox experiment -- and
    1024 independent source -> sink pairs; one persistent launch per step."""
    import torch

    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    slot_bytes = 128        # one 64-byte mailbox slot written and read per message
    out = {}
    for label, n_src, n_sink, per in (("n_to_1", 100, 1, 20_000), ("pairs", 1024, 1024, 2_000)):
        # the slot pool is max_actors x the default capacity: the sinks' size
        sink_cap = 1 << 14 if n_sink == 1 else 4096
        with C.Runtime(max_actors=n_src + n_sink, mailbox_capacity=sink_cap, scheduler=_sched(args)) as rt:
            sinks = [rt.spawn(C.SINK) for _ in range(n_sink)]
            srcs = [rt.spawn(C.SOURCE, next=sinks[i % n_sink], mailbox_capacity=4) for i in range(n_src)]
            m = np.zeros(n_src, C.DMSG_DTYPE)
            m["actor"] = np.array(srcs, np.uint32) - 1
            m["kind"] = C.SOURCE
            m["u64"] = per
            m["tag"] = np.arange(n_src)
            d_m = torch.from_numpy(m.view(np.uint8).copy()).cuda()
            d_r = torch.zeros(n_src * 32, dtype=torch.uint8, device="cuda")
            stream = torch.cuda.ExternalStream(rt.stream())
            torch.cuda.synchronize()
            for _ in range(args.warmup):
                rt.reset_actors()
                rt.request_batch_device(d_m.data_ptr(), n_src, d_r.data_ptr())
            rt.stream_sync()
            times = []
            for _ in range(args.steps):
                rt.reset_actors()
                e0, e1 = _events(stream)
                e0.record(stream)
                rt.request_batch_device(d_m.data_ptr(), n_src, d_r.data_ptr())
                e1.record(stream)
                rt.stream_sync()
                times.append(e0.elapsed_time(e1) / 1e3)
            total = sum(rt.sink_totals(s)[0] for s in sinks)
            if total != n_src * per:
                raise SystemExit(f"bench: mailbox {label}: sinks counted {total} of {n_src * per}")
            st = rt.stats()
            t = float(np.mean(times))
            msgs = n_src * per
            out[label] = {"sources": n_src, "sinks": n_sink, "messages": msgs, "ms_per_step": 1e3 * t,
                          "timing_stats": timing_stats(times, msgs),
                          "msgs_per_s": msgs / t,
                          "roofline": {"bound": "hbm", "achieved": slot_bytes * msgs / t / 1e9, "peak": hbm,
                                       "unit": "GB/s", "frac": slot_bytes * msgs / t / 1e9 / hbm,
                                       "bytes_per_msg": slot_bytes},
                          "gpu_launches": st["launches"]}
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": "mailbox: SOURCE actors streaming into SINK "
                      "actors (N:1 and pairs)", "steps": args.steps, "results": out,
                      "value": out["n_to_1"]["msgs_per_s"]}))
    return 0


FP32_OPS_PER_ITER = 8          # 3 multiplies + 5 adds per escape iteration
FP32_LANES_PER_SM = 128


def run_mandel(args):
    """Mandelbrot actors (the OpenCL actor experiment, Sec. 5): the 1920 x 1080
    image of [-0.5 - 0.7375i, 0.1 - 0.1375i] at 120 and at 1200 iterations, sent
    as one whole-image message per step (the paper's per-run time), as 100
    whole-image messages to one MANDELBROT actor (the paper's 100 runs at
    once), and as one message per row to one actor per row (1080 actors, 10
    images, 10,800 messages per step -- the one-actor-per-row split of the
    paper's CPU Mandelbrot benchmark); persistent drain against one kernel
    launch per message."""
    import torch

    import oracle
    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    Wd, Hd = W.MANDEL_WIDTH, W.MANDEL_HEIGHT
    x0, y0, dx, dy = W.mandel_image()
    peaks = measured_peaks()
    fp32_rate = C.measure_fp32_rate()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    results = {}
    clocks = ClockSampler(physical_gpu(0))
    clocks.start()
    iters = [int(x) for x in args.mandel_iters.split(",")]
    shapes = [x.strip() for x in args.mandel_shapes.split(",")]
    for max_iter in iters:
        for shape, images, rows_per_msg in (("single", 1, Hd), ("image", 100, Hd), ("row", 10, 1)):
            if shape not in shapes:
                continue
            if shape != "single":
                images = args.mandel_images or images
            per_image = Hd // rows_per_msg
            count = images * per_image
            out = torch.zeros((images, Hd, Wd), dtype=torch.int32, device="cuda")
            desc = np.zeros(count, C.MANDEL_DESC_DTYPE)
            img = np.repeat(np.arange(images), per_image)
            row0 = np.tile(np.arange(per_image) * rows_per_msg, images)
            desc["out"] = out.data_ptr() + 4 * (img.astype(np.uint64) * Hd * Wd + row0.astype(np.uint64) * Wd)
            desc["width"], desc["rows"], desc["row0"], desc["max_iter"] = Wd, rows_per_msg, row0, max_iter
            desc["x0"], desc["y0"], desc["dx"], desc["dy"] = x0, y0, dx, dy
            d_desc = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
            label = f"iter{max_iter}_{shape}"
            _note(f"mandel {label}: {count} messages")
            n_act = per_image                     # one actor per slice: 1 (whole images) or 1080 (rows)
            cap = 128 if n_act == 1 else 16
            with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=n_act, mailbox_capacity=cap) as rt:
                acts = np.array([rt.spawn(C.MANDELBROT) for _ in range(n_act)], np.uint64)
                actor_of = acts[np.tile(np.arange(per_image), images)]
                m = np.zeros(count, C.DMSG_DTYPE)
                m["actor"] = actor_of - 1
                m["kind"] = C.MANDELBROT
                m["u64"] = d_desc.data_ptr() + np.arange(count, dtype=np.uint64) * C.MANDEL_DESC_DTYPE.itemsize
                m["sender_seq"] = np.arange(count)
                m["tag"] = np.arange(count)
                d_m = torch.from_numpy(m.view(np.uint8).copy()).cuda()
                d_r = torch.zeros(count * 32, dtype=torch.uint8, device="cuda")
                stream = torch.cuda.ExternalStream(rt.stream())
                torch.cuda.synchronize()
                for _ in range(args.warmup):
                    rt.request_batch_device(d_m.data_ptr(), count, d_r.data_ptr())
                rt.stream_sync()
                rt.stats()
                times = []
                reps = max(args.steps, 20) if shape == "single" else args.steps   # sub-ms steps: more samples
                for _ in range(reps):
                    with torch.cuda.stream(stream):
                        flush.add_(1.0)
                    e0, e1 = _events(stream)
                    e0.record(stream)
                    rt.mark()
                    rt.request_batch_device(d_m.data_ptr(), count, d_r.data_ptr())
                    e1.record(stream)
                    rt.stream_sync()
                    times.append(e0.elapsed_time(e1) / 1e3)
                st = rt.stats()
                rep_ = d_r.cpu().numpy().view(C.DREPLY_DTYPE)
                if not (np.all(rep_["status"] == 0) and np.all(rep_["r0"] == rows_per_msg * Wd)):
                    raise SystemExit(f"bench: mandel {label}: replies incomplete")
                counts_sum = int(rep_["r1"][:per_image].astype(np.uint64).sum())    # one image
                sums = rep_["r1"].reshape(images, per_image).sum(axis=1)
                if not np.all(sums == counts_sum):
                    raise SystemExit(f"bench: mandel {label}: images differ")
                got = out[0].cpu().numpy().view(np.uint32)
                for j in (0, 311, 540, 777, Hd - 1):                  # sampled rows against the oracle
                    want, _ = oracle.mandel_rows(x0, y0, dx, dy, Wd, j, 1, max_iter)
                    if not np.array_equal(got[j], want[0]):
                        raise SystemExit(f"bench: mandel {label}: row {j} differs from the oracle")
                lat = (rep_["t_done"].astype(np.int64) - np.int64(st["t_mark"])) / 1e6
                t = float(np.mean(times))
                ops = FP32_OPS_PER_ITER * float(counts_sum) * images
                v = {"messages": count, "actors": n_act, "images": images, "ms_per_step": 1e3 * t,
                     "timing_stats": timing_stats(times, count),
                     "msgs_per_s": count / t,
                     "images_per_s": images / t, "mpix_per_s": images * Wd * Hd / t / 1e6,
                     "mean_iterations": counts_sum / (Wd * Hd),
                     "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                     "fp32_tops": ops / t / 1e12, "gpu_launches": st["launches"]}
                if not args.skip_per_message:
                    rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
                    ds = [C.MandelDesc(int(desc["out"][i]), Wd, rows_per_msg, int(row0[i]), max_iter,
                                       float(x0), float(y0), float(dx), float(dy)) for i in range(count)]
                    msgs = (C.Msg * count)()
                    for i in range(count):
                        msgs[i] = C.Runtime.mandel_msg(ds[i], tag=i)
                    actors = actor_of
                    rt.await_batch(rt.request_batch(actors[:per_image], msgs), timeout_ns=AWAIT_NS)   # warm-up
                    pm = []
                    for _ in range(reps if shape == "single" else max(1, min(args.steps, 3))):
                        with torch.cuda.stream(stream):
                            flush.add_(1.0)
                        e0, e1 = _events(stream)
                        torch.cuda.synchronize()
                        e0.record(stream)
                        h = rt.request_batch(actors, msgs)
                        e1.record(stream)
                        prep = rt.await_batch(h, timeout_ns=AWAIT_NS)
                        torch.cuda.synchronize()
                        pm.append(e0.elapsed_time(e1) / 1e3)
                    if not np.array_equal(prep["r1"], rep_["r1"]):
                        raise SystemExit(f"bench: mandel {label}: per-message sums differ")
                    tp = float(np.mean(pm))
                    v["per_message_launch"] = {"ms": 1e3 * tp, "msgs_per_s": count / tp,
                                               "speedup_persistent": tp / t}
                results[label] = v
            del out, d_desc
            torch.cuda.empty_cache()
    clk = clocks.stop()
    mhz = clk.get("sm_max_mhz") or 2070.0
    nominal = torch.cuda.get_device_properties(0).multi_processor_count * FP32_LANES_PER_SM * mhz * 1e6 / 1e12
    for v in results.values():
        v["roofline"] = {"bound": "alu", "achieved": v["fp32_tops"], "peak": nominal, "unit": "TFLOP/s",
                         "frac": v["fp32_tops"] / nominal, "measured_fp32_tops": fp32_rate / 1e12,
                         "frac_of_measured": v["fp32_tops"] / (fp32_rate / 1e12),
                         "note": "float32 multiplies and adds of the escape iterations (8 per iteration); "
                                 "peak = 152 SMs x 128 lanes x max SM clock"}
    # CPU baseline: the oracle on a bounded sample of rows of the large problem
    budget = min(args.cpu_seconds, 10.0)
    t0 = time.perf_counter()
    done_px = done_iter = 0
    j = 0
    while time.perf_counter() - t0 < budget and j < Hd:
        _, s_ = oracle.mandel_rows(x0, y0, dx, dy, Wd, (j * 37) % Hd, 1, 1200)
        done_px += Wd
        done_iter += s_
        j += 1
    secs = time.perf_counter() - t0
    head = results.get("iter1200_image") or next(iter(results.values()))
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Mandelbrot actor: 1920 x 1080 over [-0.5-0.7375i, 0.1-0.1375i], 120 and 1200 "
                                   "iterations; whole-image and per-row messages",
                       "l2": "flushed between steps (256 MiB write); outputs 830 MB per image step"},
            "value": head["msgs_per_s"], "ms_per_step": head["ms_per_step"], "results": results,
            "roofline": head["roofline"], "clocks": clk,
            "cpu_baseline": {"value": (done_px / (Wd * Hd)) / secs, "unit": "images/s (1200 iterations)",
                             "cores": 1, "kind": "oracle",
                             "sample": f"{j} sampled rows of the 1200-iteration image in {secs:.1f} s, one core"}}
    print(json.dumps(line))
    return 0


def run_spawn(args):
    """Actor creation (Sec. 5, "Overhead of Actor Creation"): one FORK root computes
    2^n by recursive creation, every actor spawned on the device from the pool and
    recycled; one device-resident start message per step."""
    import torch

    from oracle import actors as OA
    from paper_1505_07368_gb300 import cafgpu as C
    torch.cuda.set_device(0)
    n = args.fork_n
    spawns = (2 << n) - 2
    msgs = (4 << n) - 3                    # start and result messages per step
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # per spawned actor: its 128 B record written, one start and one result slot
    # (64 B each) written and read
    bytes_per_actor = 128 + 2 * 128
    clocks = ClockSampler(physical_gpu(0))
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=max(1 << 21, spawns),
                   scheduler=_sched(args)) as rt:
        root = rt.spawn(C.FORK)
        m = np.zeros(1, C.DMSG_DTYPE)
        m["actor"], m["kind"], m["u64"] = root - 1, C.FORK, n
        d_m = torch.from_numpy(m.view(np.uint8).copy()).cuda()
        d_r = torch.zeros(32, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.ExternalStream(rt.stream())
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            rt.request_batch_device(d_m.data_ptr(), 1, d_r.data_ptr())
        rt.stream_sync()
        rt.stats()
        clocks.start()
        times = []
        for _ in range(args.steps):
            e0, e1 = _events(stream)
            e0.record(stream)
            rt.request_batch_device(d_m.data_ptr(), 1, d_r.data_ptr())
            e1.record(stream)
            rt.stream_sync()
            times.append(e0.elapsed_time(e1) / 1e3)
        clk = clocks.stop()
        st = rt.stats()
        rep_ = d_r.cpu().numpy().view(C.DREPLY_DTYPE)
        if (rep_["status"][0], rep_["r0"][0], rep_["r1"][0]) != (0, 1 << n, spawns):
            raise SystemExit(f"bench: spawn: wrong reply {rep_}")
        if st["device_spawns"] != args.steps * spawns or st["messages"] != args.steps * msgs:
            raise SystemExit(f"bench: spawn: counters {st}")
    t = float(np.mean(times))
    # CPU baseline: the oracle's message-by-message simulation, one core, n = 16
    t0 = time.perf_counter()
    ref = OA.fork_tree(16)
    ct = time.perf_counter() - t0
    print(json.dumps({
        "metric": METRIC, "unit": "actors spawned/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"actor creation: 2^{n} by recursive spawning, {spawns} device spawns and {msgs} "
                               f"messages per step, one FORK root, pool of {max(1 << 21, spawns)} records",
                   "scheduler": args.scheduler,
                   "warps_per_team": "1 (the runtime's choice when no factor actor exists)"},
        "value": spawns / t, "ms_per_step": 1e3 * t, "timing_stats": timing_stats(times, spawns),
        "msgs_per_s": msgs / t,
        "roofline": {"bound": "hbm", "achieved": bytes_per_actor * spawns / t / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": bytes_per_actor * spawns / t / 1e9 / hbm, "bytes_per_actor": bytes_per_actor,
                     "note": "record and mailbox bytes per spawned actor; the path is bound by atomics and "
                             "queue latency, not by this traffic"},
        "gpu_launches": st["launches"], "clocks": clk,
        "cpu_baseline": {"value": ref["spawned"] / ct, "unit": "actors spawned/s", "cores": 1, "kind": "oracle",
                         "sample": f"n = 16 ({ref['spawned']} spawns) in {ct:.2f} s, message-by-message simulation"}}))
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "gemm":
        return run_gemm(args)
    if args.workload == "ring":
        return run_ring(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "mailbox":
        return run_mailbox(args)
    if args.workload == "small":
        return run_small(args)
    if args.workload == "mandel":
        return run_mandel(args)
    if args.workload == "spawn":
        return run_spawn(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
