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
SM_COUNT = 152
IMAD_PER_SM_CLK = 64          # 32-bit integer multiply(-add) lanes per SM per clock
MULS_PER_TEST = 3             # the Montgomery divisibility test: m0, n + m0*p, m1


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--factor-batch", type=int, default=16)
    ap.add_argument("--factor-warps", type=int, default=4)
    ap.add_argument("--ctas-per-sm", type=int, default=2)
    ap.add_argument("--skip-per-message", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--max-messages", type=int, default=None, help="truncate the workload (profiling)")
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
    rt = C.Runtime(max_factor_n=(1 << 56) - 1, max_actors=wl.n_actors, mailbox_capacity=512,
                   ingress_capacity=1 << 17, max_inflight_requests=1 << 17, factor_batch=args.factor_batch,
                   factor_warps=args.factor_warps, ctas_per_sm=args.ctas_per_sm)
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
    peak_tops = SM_COUNT * IMAD_PER_SM_CLK * sm_max * 1e6 / 1e12
    achieved_tops = MULS_PER_TEST * tests_alg / (dev_s / args.steps) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tmul/s",
                "frac": achieved_tops / peak_tops, "traffic": None,
                "kernel": "k_drain", "algorithmic_tests_per_step": tests_alg,
                "executed_tests_per_step": st["prime_tests"] / args.steps,
                "peak_basis": f"{SM_COUNT} SMs x {IMAD_PER_SM_CLK} IMAD/clk x {sm_max:.0f} MHz (sm_max_mhz of measured)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "messages": count, "actors": wl.n_actors,
                   "factor_batch": args.factor_batch, "factor_warps": args.factor_warps,
                   "ctas_per_sm": args.ctas_per_sm, "l2": "flushed between steps (256 MiB write)",
                   "timing": "CUDA events on the runtime stream, per step"},
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
        rrep = rt.await_batch(h)
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
        rt.await_batch(h)
        rt.sync()
        times = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = rt.request_batch(actors, msgs)
            erep = rt.await_batch(h)
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


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
