"""Benchmark: monomer insertions/s of Rosenbluth chain growth on one GB300.

A step is one pass of the whole hot path over one batch:
  lattice interacting SAW, N = 64, 10^7 chains, beta*eps = 0, 0.2, 0.4
  (seeds 2, 3, 4): growth of every chain (rosen_lattice_grow) and the FP64
  ensemble reduction of each ensemble (rosen_reduce).
value = monomer insertions ((N-1) per chain) per second over the whole job.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a
device synchronize, timed with CUDA events on the launching stream.  The
per-chain outputs (320 MB per ensemble) exceed the 129 MB L2, and the
kernels read no inputs, so no L2 flush is needed between steps.
The dominant kernel is also timed launch by launch (CUDA events on the same
stream) for the roofline figure.  --impl reference times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 64
C = 10_000_000
BETAS = [(0.0, 2), (0.2, 3), (0.4, 4)]
WORKLOAD = "lattice ISAW N=64, 1e7 chains x beta*eps {0, 0.2, 0.4}"
METRIC = "monomer insertions/s at N=64 (lattice & real space) vs roofline; served p50/p99 latency"
UNIT = "insertions/s"

# Algorithmic integer work of one lattice chain (lane operations): every
# pair test (an earlier monomer against the chain end) costs 6 operations
# (add, range test, two shift-or for the table index, table load,
# accumulate) and every step 100 (Philox4x32-10 at 70, selection and log
# at 30).  Athermal steps test only monomers of the right parity.
PAIR_OPS, STEP_OPS = 6, 100


def lattice_pairs(N, athermal):
    if athermal:
        return sum(i // 2 for i in range(2, N))
    return (N - 1) * (N - 2) // 2


def lattice_ops_per_chain(N, athermal):
    return PAIR_OPS * lattice_pairs(N, athermal) + STEP_OPS * (N - 1)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sms, mhz = 152, 2070.0
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return sms, mhz


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_04381_gb300 import rosen

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    stream = torch.cuda.current_stream()
    # Weak scaling: every rank grows its own C chains (global chain indices
    # rank*C .. rank*C + C - 1 of each ensemble); no data-path collective.
    chain0 = rank * C
    outs = [rosen.lattice_outputs(N, C, device=dev) for _ in BETAS]
    params = [rosen.lattice_params(seed, N, C, beta_eps=b, chain0=chain0) for b, seed in BETAS]
    stats = [rosen.stats_tensor(dev) for _ in BETAS]
    ws = rosen.reduce_workspace(C, dev)
    rins = [rosen.lattice_reduce_in(o, N, use_counts=int(b == 0.0)) for o, (b, _) in zip(outs, BETAS)]
    launches_per_step = len(BETAS) * 3          # growth + two reduction kernels each

    kernel_ev = []

    def step(record=False):
        for q in range(len(BETAS)):
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            rosen.rosen_lattice_grow(params[q], outs[q], stream)
            if record:
                e1.record(stream)
                kernel_ev.append((q, e0, e1))
            rosen.rosen_reduce(rins[q], stats[q], ws, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    ins_per_step = len(BETAS) * C * (N - 1) * world
    value = ins_per_step / (ms_per_step / 1e3)

    # Roofline of the dominant kernel (interacting growth, beta*eps > 0).
    per_q = {q: [] for q in range(len(BETAS))}
    for q, e0, e1 in kernel_ev:
        per_q[q].append(e0.elapsed_time(e1))
    sms, mhz = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_lane_ops = sms * 128 * mhz * 1e6
    isaw_ms = statistics.mean(per_q[1] + per_q[2])
    ath_ms = statistics.mean(per_q[0])
    achieved = lattice_ops_per_chain(N, False) * C / (isaw_ms / 1e3)
    parts = {
        "lattice_athermal_ms": ath_ms,
        "lattice_isaw_ms": isaw_ms,
        "lattice_athermal_ins_per_s": C * (N - 1) / (ath_ms / 1e3),
        "lattice_isaw_ins_per_s": C * (N - 1) / (isaw_ms / 1e3),
    }

    e2e = measure_e2e(args, rosen, torch, dev, stream, chain0, world)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (Philox-seeded growth; no input data)",
        "config": {"workload": WORKLOAD, "N": N, "chains_per_ensemble": C * world,
                   "beta_eps": [b for b, _ in BETAS], "seeds": [s for _, s in BETAS],
                   "l2": "no inputs; outputs 320 MB per ensemble > 129 MB L2, no flush",
                   "parallelism": "dp%d (chain ranges per GPU)" % world},
        "parts": parts,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_lane_ops / 1e12,
                     "unit": "Tops/s (32-bit lane ops)", "frac": achieved / peak_lane_ops,
                     "traffic": None, "kernel": "lattice_lane_kernel<isaw>",
                     "ops_per_chain": lattice_ops_per_chain(N, False),
                     "peak_basis": "%d SMs x 128 lanes x %.0f MHz (max SM clock)" % (sms, mhz)},
        "clocks": clocks.summary(),
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)


def measure_e2e(args, rosen, torch, dev, stream, chain0, world):
    """Same metric through the C ABI with host buffers: per step the per-chain
    outputs (log W, R^2, N^2 R_g^2) and the statistics are copied back to
    pinned host memory; the only host-to-device input is the parameter block."""
    outs = [rosen.lattice_outputs(N, C, device=dev) for _ in BETAS]
    host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
             for k, v in o.items() if k != "counts"} for o in outs]
    stats = [rosen.stats_tensor(dev) for _ in BETAS]
    hstats = [torch.empty(len(rosen.STAT_KEYS), dtype=torch.float64, pin_memory=True)
              for _ in BETAS]
    ws = rosen.reduce_workspace(C, dev)
    d2h = sum(v.numel() * v.element_size() for h in host for v in h.values()) + \
        sum(h.numel() * 8 for h in hstats)
    h2d = len(BETAS) * 48

    def step():
        for q, (b, seed) in enumerate(BETAS):
            p = rosen.lattice_params(seed, N, C, beta_eps=b, chain0=chain0)
            rosen.rosen_lattice_grow(p, outs[q], stream)
            rosen.rosen_reduce(rosen.lattice_reduce_in(outs[q], N, int(b == 0.0)), stats[q], ws,
                               stream)
            for k in host[q]:
                host[q][k].copy_(outs[q][k], non_blocking=True)
            hstats[q].copy_(stats[q], non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(1, args.warmup)):
        step()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = (time.perf_counter() - t0) / steps
    return {"value": len(BETAS) * C * (N - 1) / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def oracle_sample(threads):
    """The oracle on a bounded sample: the first S chains of each ensemble."""
    import oracle
    S = int(os.environ.get("ROSEN_CPU_SAMPLE", "600000"))
    t0 = time.perf_counter()
    for b, seed in BETAS:
        oracle.lattice_run(seed, N, S, beta_eps=b, threads=threads)
    dt = time.perf_counter() - t0
    return len(BETAS) * S * (N - 1) / dt, dt, S


def cpu_baseline(args):
    import oracle
    threads = oracle.default_threads()
    v, dt, S = oracle_sample(threads)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "first %d chains of each of the 3 ensembles (%.1f s)" % (S, dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    threads = oracle.default_threads()
    for _ in range(args.warmup):
        pass
    times = []
    v = None
    for _ in range(max(1, args.steps)):
        v, dt, S = oracle_sample(threads)
        times.append(dt)
    v = len(BETAS) * S * (N - 1) / statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "N": N},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "first %d chains of each of the 3 ensembles per step" % S},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        os.environ.setdefault("ROSEN_CPU_SAMPLE", "200000")
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
