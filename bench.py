"""Benchmark: monomer insertions/s of Rosenbluth chain growth on one GB300.

A step is one pass of the whole hot path over one batch of synthetic chains:
  lattice interacting SAW, N = 64, 10^7 chains, beta*eps = 0, 0.2, 0.4
  (seeds 2, 3, 4), and real-space hard spheres, N = 64, k = 32 trial
  directions, bond = diameter = 1, 10^7 chains (seed 5): growth of every
  chain (rosen_lattice_grow / rosen_offlattice_grow) and the FP64 ensemble
  reduction of each ensemble (rosen_reduce).
value = monomer insertions ((N-1) per chain) per second over the whole step;
"parts" gives each ensemble's own rate.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a
device synchronize, timed with CUDA events on the launching stream.  The
kernels read no inputs and the per-chain outputs (160-320 MB per ensemble)
exceed the 129 MB L2, so no L2 flush is needed between steps.  Every growth
launch is also timed with its own pair of CUDA events on the same stream for
the roofline figure.  --impl reference times the FP64 CPU oracle instead, on a
bounded sample of the same workload.
"""
import argparse
import ctypes
import json
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
K_TRIALS = 32
REAL_POT = "hard_sphere"    # the step's real-space ensemble: hard_sphere or lj
REAL_BETA = 0.0
LATTICE = [(0.0, 2), (0.2, 3), (0.4, 4)]
HS_SEED = 5
WORKLOAD = ("N=64, 1e7 chains per ensemble: lattice ISAW beta*eps {0, 0.2, 0.4} + "
            "real-space hard spheres k=32")
METRIC = "monomer insertions/s at N=64 (lattice & real space) vs roofline; served p50/p99 latency"
UNIT = "insertions/s"

# Roofline work per chain, counted for the brute-force method, which tests
# every earlier monomer against every trial.
#  lattice: (N-1)(N-2)/2 pair tests at 7 INT ops, a 70-op Philox call and 30
#    ops of selection and log per step (20,000 ops/chain at N = 64);
#  real space: k (N-1)(N-2)/2 pair tests at 8 FP32 ops, and per step k
#    Philox calls and directions at 90 ops (~6.8e5 ops/chain at N = 64, k = 32).
BRUTE_LAT_PAIR, BRUTE_LAT_STEP = 7, 100
BRUTE_OFF_PAIR, BRUTE_OFF_TRIAL = 8, 90

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant growth -- hard spheres, N = 64, k = 32, 10^7 chains, both
# passes -- from one ncu capture of that launch: first pass 23,213,312 +
# 78,660,864, second pass 18,835,968 + 17,702,912.  Reported as the
# roofline's traffic for that configuration only.
HS_TRAFFIC_BYTES = 22961664 + 78489856 + 18875648 + 18076160


def brute_lattice_ops(N):
    return BRUTE_LAT_PAIR * (N - 1) * (N - 2) // 2 + BRUTE_LAT_STEP * (N - 1)


def brute_offlattice_ops(N, k):
    return BRUTE_OFF_PAIR * k * (N - 1) * (N - 2) // 2 + BRUTE_OFF_TRIAL * k * (N - 1)


# Work the kernels actually execute, in 32-bit lane operations (they test only
# the monomers that can reach a trial):
#  lattice: 6 per pair test (add, range test, gather multiply, shift, table
#    load, accumulate), 100 per step (Philox 70, selection and log 30);
#    athermal steps test only monomers of the matching parity;
#  real space: 10 per bead scanned for the near list, 4 per pair test
#    (3 FMA + min) of a listed bead against a trial, 60 per trial per step
#    (half a Philox call, the direction), 40 per step (selection, commit).
LAT_PAIR_OPS, LAT_STEP_OPS = 6, 100
OFF_SCAN_OPS, OFF_PAIR_OPS, OFF_TRIAL_OPS, OFF_STEP_OPS = 10, 4, 60, 40


def lattice_pairs(N, athermal):
    if athermal:
        return sum(i // 2 for i in range(2, N))
    return (N - 1) * (N - 2) // 2


def lattice_ops_per_chain(N, athermal):
    return LAT_PAIR_OPS * lattice_pairs(N, athermal) + LAT_STEP_OPS * (N - 1)


def offlattice_ops(N, k, chains, listed):
    scanned = chains * (N - 1) * (N - 2) // 2
    return (OFF_SCAN_OPS * scanned + OFF_PAIR_OPS * k * listed +
            (OFF_TRIAL_OPS * k + OFF_STEP_OPS) * (N - 1) * chains)


def measured_peak(key, fallback):
    """A figure of the measured peaks file (fallback when it is missing)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f).get(key, fallback))
    return fallback


def sm_max_mhz():
    return measured_peak("sm_max_mhz", 2070.0)


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
                 "--format=csv,noheader,nounits", "-lms", "100"],
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


class Ensembles:
    """The step's ensembles: parameters, output tensors, reduction inputs."""

    def __init__(self, rosen, torch, dev, chain0, with_hs=True, max_attempts=0):
        self.rosen = rosen
        self.items = []
        restart = max_attempts > 1
        for b, seed in LATTICE:
            out = rosen.lattice_outputs(N, C, device=dev, attempts=restart)
            self.items.append({
                "name": "lattice_beps%.1f" % b, "kind": "lattice", "athermal": b == 0.0,
                "params": rosen.lattice_params(seed, N, C, beta_eps=b, chain0=chain0,
                                               max_attempts=max_attempts),
                "out": out, "rin": rosen.lattice_reduce_in(out, N, use_counts=int(b == 0.0)),
                "stats": rosen.stats_tensor(dev)})
        if with_hs:
            out = rosen.offlattice_outputs(N, C, device=dev, counters=True, attempts=restart)
            pot = rosen.ROSEN_LJ if REAL_POT == "lj" else rosen.ROSEN_HARD_SPHERE
            self.items.append({
                "name": "%s_k%d" % (REAL_POT, K_TRIALS), "kind": "offlattice",
                "params": rosen.offlattice_params(HS_SEED, N, C, K_TRIALS, potential=pot,
                                                  beta_eps=REAL_BETA, chain0=chain0,
                                                  max_attempts=max_attempts),
                "out": out, "rin": rosen.offlattice_reduce_in(out, N, K_TRIALS),
                "stats": rosen.stats_tensor(dev)})
        self.ws = rosen.reduce_workspace(C, dev)

    def grow(self, it, stream):
        if it["kind"] == "lattice":
            self.rosen.rosen_lattice_grow(it["params"], it["out"], stream)
        else:
            self.rosen.rosen_offlattice_grow(it["params"], it["out"], stream)

    def reduce(self, it, stream):
        self.rosen.rosen_reduce(it["rin"], it["stats"], self.ws, stream)

    def launches_per_step(self):
        # Growth and two reduction kernels per ensemble; hard spheres grow in
        # two passes (growth, then the deferred chains).
        return sum(4 if it["kind"] == "offlattice" and REAL_POT == "hard_sphere" else 3
                   for it in self.items)


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
    # Weak scaling: every rank grows its own C chains of each ensemble (global
    # chain indices rank*C .. rank*C + C - 1); no data-path collective.
    chain0 = rank * C
    ens = Ensembles(rosen, torch, dev, chain0, with_hs=not args.lattice_only,
                    max_attempts=args.max_attempts)
    kernel_ev = []

    def step(record=False):
        for q, it in enumerate(ens.items):
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            ens.grow(it, stream)
            if record:
                e1.record(stream)
                kernel_ev.append((q, e0, e1))
            ens.reduce(it, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for it in ens.items:
        if "counters" in it["out"]:
            it["out"]["counters"].zero_()
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
    from paper_1704_04381_gb300 import shard
    if world > 1:
        ms = shard.max_over_ranks(ms)
    ms_per_step = ms / args.steps
    ins_per_step = len(ens.items) * C * (N - 1) * world
    value = ins_per_step / (ms_per_step / 1e3)

    per_q = {q: [] for q in range(len(ens.items))}
    for q, e0, e1 in kernel_ev:
        per_q[q].append(e0.elapsed_time(e1))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_max_mhz()
    peak = sms * 128 * mhz * 1e6
    parts = {}
    rooflines = []
    for q, it in enumerate(ens.items):
        kms = statistics.mean(per_q[q])
        st = rosen.stats_dict(it["stats"])
        if world > 1:
            # Every rank grew its own chain range: merge the statistics (18
            # numbers per rank) into the ensemble's.
            st = shard.gather_stats(st, N, K_TRIALS if it["kind"] == "offlattice" else 0)
        part = {"kernel_ms": kms, "insertions_per_s": C * (N - 1) / (kms / 1e3),
                "mean_r2": st["mean_r2"], "se_r2": st["se_r2"], "logZ": st["logZ"],
                "n_alive": st["n_alive"], "growths": st["n"]}
        if it["kind"] == "lattice":
            ops = lattice_ops_per_chain(N, it["athermal"]) * C
            sops = brute_lattice_ops(N) * C
            kname = "lattice_lane_kernel<%s>" % ("athermal" if it["athermal"] else "isaw")
        else:
            cnt = it["out"]["counters"].cpu().tolist()
            reps = max(1, args.steps)
            listed = cnt[2] / reps
            ops = offlattice_ops(N, K_TRIALS, C, listed)
            sops = brute_offlattice_ops(N, K_TRIALS) * C
            part.update({"fp64_redecided_steps": cnt[0] / reps,
                         "listed_beads_per_step": listed / (C * (N - 1))})
            kname = ("offlattice_queue_kernel<16,2,hard sphere,defer> + offlattice_deferred_kernel"
                     if REAL_POT == "hard_sphere"
                     else "offlattice_queue_kernel<LJ, k=%d, beta eps %g>" % (K_TRIALS, REAL_BETA))
        part["ops_per_chain"] = ops / C
        part["brute_ops_per_chain"] = sops / C
        # Brute-force pair tests per second (every earlier monomer against
        # every trial; the lattice scores six neighbours with one test).
        pairs = (N - 1) * (N - 2) // 2 * (1 if it["kind"] == "lattice" else K_TRIALS)
        part["pair_tests_per_s"] = pairs * C / (kms / 1e3)
        parts[it["name"]] = part
        rooflines.append((kms, sops, ops, kname))
    kms, sops, ops, kname = max(rooflines)
    launches = ens.launches_per_step() * args.steps
    achieved = sops / (kms / 1e3)
    executed = ops / (kms / 1e3)

    # The small correctness configuration, timed too: athermal lattice chains,
    # N = 16, 10^5 chains, seed 1 (growth and reduction, CUDA events).
    n16 = None
    if rank == 0:
        o16 = rosen.lattice_outputs(16, 100_000, device=dev)
        p16 = rosen.lattice_params(1, 16, 100_000)
        r16 = rosen.lattice_reduce_in(o16, 16, use_counts=1)
        s16, w16 = rosen.stats_tensor(dev), rosen.reduce_workspace(100_000, dev)
        for _ in range(3):
            rosen.rosen_lattice_grow(p16, o16, stream)
            rosen.rosen_reduce(r16, s16, w16, stream)
        a16, b16 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a16.record(stream)
        for _ in range(20):
            rosen.rosen_lattice_grow(p16, o16, stream)
            rosen.rosen_reduce(r16, s16, w16, stream)
        b16.record(stream)
        torch.cuda.synchronize()
        ms16 = a16.elapsed_time(b16) / 20
        n16 = {"workload": "lattice athermal N=16, 1e5 chains, seed 1", "ms": ms16,
               "insertions_per_s": 100_000 * 15 / (ms16 / 1e3),
               "logZ": rosen.stats_dict(s16)["logZ"]}
    e2e = None if args.no_e2e else measure_e2e(args, rosen, torch, dev, stream, chain0, ens, world)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    # The batched and served configurations and the conformation-store run
    # (one GPU only): the metric's latency half and the batched/served
    # throughput next to the single-ensemble path.
    batched = served5 = served_ok = stored = perm = None
    if world == 1 and not (args.no_served and args.no_batched and args.no_store_coords and
                           args.no_perm):
        del ens
        torch.cuda.empty_cache()
        if not args.no_perm:
            perm = perm_leg(rosen, torch)
            torch.cuda.empty_cache()
        if not args.no_store_coords:
            stored = store_coords_leg(rosen, torch)
        if not args.no_batched:
            batched = batched_leg(rosen, torch)
        if not args.no_served:
            sf = args.served_policy == "shortest_first"
            served5 = served_run(rosen, 2000.0, args.served_duration, 40.0, 256, 1.0,
                                 shortest_first=sf, replay_every=5, torch=torch)
            # The sustainable rate: 0.7 x the GPU's capacity for the offered
            # mix (requests completed under saturation are the smaller ones,
            # so their rate overstates it).
            cap, ncap = offered_capacity(rosen, torch)
            served_ok = served_run(rosen, max(1.0, 0.7 * cap), args.served_duration, 40.0, 256,
                                   1.0, shortest_first=sf, replay_every=5, torch=torch)
            if "single_path" in served_ok:
                # Below saturation the ratio is the share of the wall time the
                # single path would keep the GPU busy, not a throughput ratio.
                sp = served_ok["single_path"]
                sp["gpu_busy_fraction"] = sp.pop("served_over_single")
            served_ok["capacity_requests_per_s"] = cap
            served_ok["capacity_basis"] = ("1 / mean time alone of %d requests of the offered "
                                           "mix (every 17th of the arrival pool)" % ncap)
            served_ok["completed_per_s_under_saturation"] = (served5["completed"] /
                                                             served5["wall_s"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+fp32",
        "data": "synthetic (Philox-seeded growth; no input data)",
        "config": step_config(world, args.max_attempts),
        "parts": parts,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "Tops/s (32-bit lane ops)", "frac": achieved / peak,
                     "traffic": (HS_TRAFFIC_BYTES if (REAL_POT == "hard_sphere" and C == 10_000_000
                                                      and K_TRIALS == 32 and args.max_attempts <= 1
                                                      and "hard sphere" in kname) else None),
                     "traffic_unit": "DRAM bytes per launch (ncu, both passes)",
                     "kernel": kname, "ops_per_chain": sops / C,
                     "ops_basis": "brute-force work: every earlier monomer tested against every trial",
                     "executed_ops_per_chain": ops / C, "executed_frac": executed / peak,
                     "peak_basis": "%d SMs x 128 lanes x %.0f MHz (max SM clock)" % (sms, mhz)},
        "clocks": clocks.summary(),
        "e2e": e2e,
        "gpu_launches": launches,
        "batched": batched,
        "served_config5": served5,
        "served_sustainable": served_ok,
        "store_coords": stored,
        "perm": perm,
        "small_config": n16,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(not args.lattice_only)
    print(json.dumps(line), flush=True)


def measure_e2e(args, rosen, torch, dev, stream, chain0, ens, world=1):
    """The same metric through the C ABI with host buffers: per step the
    per-chain results (log W, R^2, R_g^2) and the statistics of every ensemble
    are copied back to pinned host memory; the only host-to-device input is
    the parameter block of each call.  Each ensemble's copies run on a second
    stream, after its reduction, while the next ensemble grows."""
    host = []
    d2h = 0
    for it in ens.items:
        h = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
             for k, v in it["out"].items() if k in ("logw", "r2", "n2rg2", "rg2")}
        hs = torch.empty(len(rosen.STAT_KEYS), dtype=torch.float64, pin_memory=True)
        host.append((h, hs))
        d2h += sum(v.numel() * v.element_size() for v in h.values()) + hs.numel() * 8
    h2d = sum(ctypes.sizeof(it["params"]) for it in ens.items)

    copier = torch.cuda.Stream(device=dev)

    def step():
        for it, (h, hs) in zip(ens.items, host):
            ens.grow(it, stream)
            ens.reduce(it, stream)
            done = torch.cuda.Event()
            done.record(stream)
            copier.wait_event(done)
            with torch.cuda.stream(copier):
                for k in h:
                    h[k].copy_(it["out"][k], non_blocking=True)
                hs.copy_(it["stats"], non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    steps = max(1, min(args.steps, 5))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = (time.perf_counter() - t0) / steps
    if world > 1:
        # The whole job: every rank's chains over the slowest rank's time.
        from paper_1704_04381_gb300 import shard
        dt = shard.max_over_ranks(dt)
    return {"value": len(ens.items) * C * (N - 1) * world / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d * world, "d2h_bytes_per_step": d2h * world}


def oracle_rates(with_hs, threads, budget_s):
    """Oracle insertion rates per ensemble kind on bounded samples."""
    import oracle
    n_lat = int(os.environ.get("ROSEN_CPU_LATTICE_SAMPLE", "0")) or None
    n_hs = int(os.environ.get("ROSEN_CPU_HS_SAMPLE", "0")) or None
    rates, notes = {}, []
    # Calibrate on a small batch, then size the sample to the time budget.
    for b, seed in LATTICE:
        t = time.perf_counter()
        oracle.lattice_run(seed, N, 2000, beta_eps=b, threads=threads)
        cal = (time.perf_counter() - t) / 2000
        S = n_lat or max(2000, int(budget_s / (len(LATTICE) + 2) / max(cal, 1e-9)))
        t = time.perf_counter()
        oracle.lattice_run(seed, N, S, beta_eps=b, threads=threads)
        dt = time.perf_counter() - t
        rates["lattice_beps%.1f" % b] = S * (N - 1) / dt
        notes.append("lattice beta_eps=%.1f: first %d chains (%.1f s)" % (b, S, dt))
    if with_hs:
        t = time.perf_counter()
        pot = oracle.LJ if REAL_POT == "lj" else oracle.HARD_SPHERE
        oracle.offlattice_run(HS_SEED, N, 200, K_TRIALS, potential=pot, beta_eps=REAL_BETA,
                              threads=threads)
        cal = (time.perf_counter() - t) / 200
        S = n_hs or max(200, int(2 * budget_s / (len(LATTICE) + 2) / max(cal, 1e-9)))
        t = time.perf_counter()
        oracle.offlattice_run(HS_SEED, N, S, K_TRIALS, potential=pot, beta_eps=REAL_BETA,
                              threads=threads)
        dt = time.perf_counter() - t
        rates["%s_k%d" % (REAL_POT, K_TRIALS)] = S * (N - 1) / dt
        notes.append("hard spheres k=32: first %d chains (%.1f s)" % (S, dt))
    # The whole step at these rates: total insertions / total time.
    total_time = sum(C * (N - 1) / r for r in rates.values())
    value = len(rates) * C * (N - 1) / total_time
    return value, rates, "; ".join(notes)


def cpu_baseline(with_hs):
    import oracle
    threads = oracle.default_threads()
    value, rates, note = oracle_rates(with_hs, threads, budget_s=15.0)
    # One core as well (the paper's CPU timings are single-core).
    v1, r1, n1 = oracle_rates(with_hs, 1, budget_s=4.0)
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": note + "; value = the full step's insertions over the summed time "
                             "at these rates", "parts": rates,
            "single_core": {"value": v1, "cores": 1, "parts": r1, "sample": n1}}


def step_config(world, max_attempts=0):
    """The step's workload description, the same for both arms."""
    return {"workload": WORKLOAD, "N": N, "chains_per_ensemble": C * world,
            "lattice_beta_eps": [b for b, _ in LATTICE], "hs_k": K_TRIALS,
            "real_space": {"potential": REAL_POT, "k": K_TRIALS, "beta_eps": REAL_BETA},
            "max_attempts": max(1, max_attempts),
            "l2": "no inputs; outputs 160-320 MB per ensemble > 129 MB L2, no flush",
            "parallelism": "dp%d (chain ranges per GPU)" % world}


def oracle_step(S, chain0, threads):
    """One scaled-down step of the oracle: the first S chains (from chain0) of
    every ensemble of the step, grown and reduced; returns the seconds taken."""
    import oracle
    t = time.perf_counter()
    for b, seed in LATTICE:
        o = oracle.lattice_run(seed, N, S, beta_eps=b, chain0=chain0, threads=threads)
        oracle.reduce(o["logw"], o["r2"].astype("float64"), o["n2rg2"] / float(N * N), N)
    pot = oracle.LJ if REAL_POT == "lj" else oracle.HARD_SPHERE
    o = oracle.offlattice_run(HS_SEED, N, S, K_TRIALS, potential=pot, beta_eps=REAL_BETA,
                              chain0=chain0, threads=threads)
    oracle.reduce(o["logw"], o["r2"], o["rg2"], N, K_TRIALS)
    return time.perf_counter() - t


def run_reference(args):
    """The oracle, unmodified, on the machine's host cores.  Each step is the
    step's workload scaled down to S chains per ensemble (the same four
    ensembles, grown and reduced), S sized so that a step takes about
    min(3 s, 60 s / steps); successive steps take successive chain ranges.
    value = the sampled insertions over the measured time, which is the full
    step's rate because the ensemble mix is the same."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    threads = oracle.default_threads()
    target = min(3.0, 60.0 / max(1, args.steps))
    cal = oracle_step(2000, 0, threads) / 2000
    S = max(2000, int(target / max(cal, 1e-9)))
    for w in range(args.warmup):
        oracle_step(max(2000, S // 4), w * S, threads)
    times = []
    for q in range(max(1, args.steps)):
        times.append(oracle_step(S, (q + 1) * S, threads))
    t_step = statistics.mean(times)
    ins_step = (len(LATTICE) + 1) * S * (N - 1)
    v = ins_step / t_step
    full_ms = 1e3 * (len(LATTICE) + 1) * C * (N - 1) / v
    note = ("per step: chains [q S, (q+1) S) of each of the %d ensembles, S = %d (%.2f%% of "
            "the 1e7 chains), grown and reduced by the oracle on %d threads"
            % (len(LATTICE) + 1, S, 100.0 * S / C, threads))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Philox-seeded growth; no input data)",
        "config": step_config(world, args.max_attempts),
        "sampled": {"chains_per_ensemble_per_step": S, "insertions_per_step": ins_step,
                    "ms_per_step_measured": 1e3 * t_step,
                    "full_step_ms_extrapolated": full_ms,
                    "note": "ms_per_step is the measured time of the sampled step; the full "
                            "1e7-chain step would take full_step_ms_extrapolated at this rate"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": note},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Batched and served modes (not part of the default step).
# ---------------------------------------------------------------------------
def batch_config(rosen, n_ens=256, seed=4, scale=1.0):
    """The batched configuration: 256 ensembles, N uniform in [8, 256], chain
    counts log-uniform in [1e3, 1e6], alternating lattice ISAW (beta eps in
    [0, 0.5]) and Lennard-Jones beads (sigma 1, cutoff 2.5, beta eps in [0, 1],
    k in {16, 32, 64}); seeds 1000 + e; drawn with numpy's default_rng(seed)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ens = []
    for e in range(n_ens):
        N = int(rng.integers(8, 257))
        C = max(1, int(10 ** rng.uniform(3, 6) * scale))
        if e % 2 == 0:
            ens.append(rosen.ensemble(rosen.ROSEN_MODEL_LATTICE, N, C, 1000 + e, e,
                                      beta_eps=float(rng.uniform(0, 0.5))))
        else:
            ens.append(rosen.ensemble(rosen.ROSEN_MODEL_OFFLATTICE, N, C, 1000 + e, e,
                                      k=int(rng.choice([16, 32, 64])), potential=rosen.ROSEN_LJ,
                                      beta_eps=float(rng.uniform(0, 1))))
    return ens


def batched_leg(rosen, torch, scale=1.0, steps=3, warmup=1):
    """The batched configuration as one graph launch per step (after tuning),
    next to the same ensembles grown and reduced one after another through
    the single-ensemble entry points.  Returns a dict (times in ms)."""
    ens = batch_config(rosen, scale=scale)
    ins = sum(e.C * (e.N - 1) for e in ens)
    b = rosen.RosenBatch(ens)
    t = time.perf_counter()
    b.tune()
    tune_s = time.perf_counter() - t
    stream = torch.cuda.current_stream()
    for _ in range(max(1, warmup)):
        b.run(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        e0.record(stream)
        for _ in range(steps):
            b.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / steps
    # The plain single-ensemble path on the same ensembles, one after another.
    outs = {}
    ws = rosen.reduce_workspace(max(e.C for e in ens))
    st = rosen.stats_tensor()

    def singles():
        for i, e in enumerate(ens):
            if e.model == rosen.ROSEN_MODEL_LATTICE:
                o = outs.get(i) or rosen.lattice_outputs(e.N, e.C)
                rosen.rosen_lattice_grow(rosen.lattice_params(e.seed, e.N, e.C, beta_eps=e.beta_eps,
                                                              ensemble=e.ensemble), o, stream)
                rosen.rosen_reduce(rosen.lattice_reduce_in(o, e.N, int(e.beta_eps == 0.0)), st, ws,
                                   stream)
            else:
                o = outs.get(i) or rosen.offlattice_outputs(e.N, e.C)
                rosen.rosen_offlattice_grow(
                    rosen.offlattice_params(e.seed, e.N, e.C, e.k, potential=e.potential,
                                            beta_eps=e.beta_eps, ensemble=e.ensemble), o, stream)
                rosen.rosen_reduce(rosen.offlattice_reduce_in(o, e.N, e.k), st, ws, stream)
            outs[i] = o
    singles()
    torch.cuda.synchronize()
    e0.record(stream)
    singles()
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1)
    cnt = b.counters().cpu().tolist()
    classes = json.loads(b.describe())
    b.close()
    del outs
    torch.cuda.empty_cache()
    return {"workload": "256 ensembles: N~U{8..256}, C log-uniform [1e3,1e6] x %g, lattice ISAW "
                        "beta eps U[0,0.5] / LJ k in {16,32,64} beta eps U[0,1]; "
                        "numpy default_rng(4)" % scale,
            "chains": sum(e.C for e in ens), "insertions": ins,
            "graph_launch_ms": batch_ms, "graph_launches_timed": steps,
            "insertions_per_s": ins / (batch_ms / 1e3),
            "single_ensemble_path_ms": single_ms,
            "single_insertions_per_s": ins / (single_ms / 1e3),
            "batched_over_single": single_ms / batch_ms, "tune_s": tune_s,
            "fp64_redecided_steps_total": cnt[0], "classes": len(classes),
            "clocks": clocks.summary()}


PERM_CFG = dict(N=64, M0=1_000_000, cap=4_000_000, mu=4.684, c_hi=3.0, c_lo=1.0 / 3.0, seed=9)


def perm_leg(rosen, torch, steps=3, warmup=1):
    """PERM (breadth first) on the cubic lattice: athermal N = 64, 10^6 chains
    started, population cap 4x10^6, thresholds 3 mu^i and mu^i / 3 with
    mu = 4.684.  value = chain steps grown per second (every chain of the
    population before step i makes one step).  Algorithmic bytes per step of
    a chain: the scan of its earlier monomers of matching parity (4 B each),
    the new monomer's key (4 B), its weight read and written (24 B) and its
    place in the population read and written (8 B), against the measured HBM
    bandwidth.  The keys an enrichment copy takes are not counted (the
    outputs do not say how many copies were made), so the figure is a lower
    bound."""
    c = PERM_CFG
    N, M0, cap = c["N"], c["M0"], c["cap"]
    p = rosen.perm_params(c["seed"], N, M0, cap, mu=c["mu"], c_hi=c["c_hi"], c_lo=c["c_lo"])
    out = rosen.perm_outputs(N, cap)
    ws = rosen.perm_workspace(N, cap)
    stream = torch.cuda.current_stream()
    for _ in range(max(1, warmup)):
        rosen.rosen_perm_run(p, out, ws, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rosen.rosen_perm_run(p, out, ws, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pop = out["population"].cpu().tolist()
    logz = out["logz"].cpu().tolist()
    grown = sum(pop[i - 1] for i in range(1, N))
    nbytes = sum(pop[i - 1] * (4 * (i // 2) + 4 + 24 + 8) for i in range(1, N))
    peak = measured_peak("hbm_gbs", 6800.0)
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"workload": "PERM athermal N=64, M0=1e6 chains started, cap 4e6, mu=4.684, "
                        "c_hi=3, c_lo=1/3, seed 9",
            "ms": ms, "chain_steps": grown, "chain_steps_per_s": grown / (ms / 1e3),
            "population_final": pop[-1], "population_max": max(pop),
            "logZ_N": logz[-1], "launches_per_run": 3 * (N - 1) + 2,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None,
                         "basis": "per chain step: 4 B per scanned key (parity), 4 B new key, "
                                  "24 B weight (read + write), 8 B slot number (read + write); "
                                  "enrichment copies not counted (lower bound)"}}


def run_perm(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_04381_gb300 import rosen
    torch.cuda.set_device(0)
    r = perm_leg(rosen, torch, steps=args.steps, warmup=args.warmup)
    line = {"metric": "PERM chain steps/s (breadth first, cubic lattice)",
            "value": r["chain_steps_per_s"], "unit": "chain steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
            "higher_is_better": True, "dtype": "int32+fp64", "data": "synthetic",
            "config": {"workload": r["workload"]}, "perm": r}
    print(json.dumps(line), flush=True)


def run_store(args):
    """Config 3 with conformations written out (chains from --chains)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_04381_gb300 import rosen
    torch.cuda.set_device(0)
    r = store_coords_leg(rosen, torch, steps=args.steps)
    line = {"metric": "real-space hard spheres N=64 k=32 with conformations stored: write GB/s",
            "value": r["write_gb_per_s"], "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "ms_per_step": r["ms"], "higher_is_better": True, "dtype": "fp32",
            "data": "synthetic", "config": {"workload": r["workload"], "chains": C},
            "store_coords": r}
    print(json.dumps(line), flush=True)


def run_batched(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_04381_gb300 import rosen
    torch.cuda.set_device(0)
    r = batched_leg(rosen, torch, scale=args.batch_scale, steps=args.steps, warmup=args.warmup)
    line = {
        "metric": "batched monomer insertions/s (256 mixed ensembles, one graph launch)",
        "value": r["insertions_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["graph_launch_ms"], "higher_is_better": True,
        "dtype": "int32+fp32", "data": "synthetic",
        "config": {"workload": r["workload"], "chains": r["chains"],
                   "insertions": r["insertions"]},
        "batched": r,
    }
    print(json.dumps(line), flush=True)


def store_coords_leg(rosen, torch, steps=2):
    """Config 3 with its conformations written out: real-space hard spheres,
    N = 64, k = 32, 10^7 chains, ROSEN_STORE_COORDS (12 B per bead per chain,
    7.7 GB per launch).  Reports the launch time against the same launch
    without the conformations, and the write bandwidth against the measured
    HBM peak."""
    stream = torch.cuda.current_stream()
    res = {}
    for flags, name in ((0, "no_coords"), (rosen.ROSEN_STORE_COORDS, "coords")):
        out = rosen.offlattice_outputs(N, C, coords=bool(flags))
        p = rosen.offlattice_params(HS_SEED, N, C, 32, flags=flags)
        rosen.rosen_offlattice_grow(p, out, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            rosen.rosen_offlattice_grow(p, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / steps
        del out
        torch.cuda.empty_cache()
    written = 12 * N * C
    peak = measured_peak("hbm_gbs", 6800.0)
    gbs = written / (res["coords"] / 1e3) / 1e9
    return {"workload": "real-space hard spheres N=64 k=32, %d chains, conformations stored" % C,
            "ms": res["coords"], "ms_without_coords": res["no_coords"],
            "coords_bytes_per_launch": written,
            "write_gb_per_s": gbs, "hbm_peak_gb_per_s": peak,
            "hbm_frac": gbs / peak,
            "basis": "12 B per bead per chain (FP32 x, y, z) written once; the kernel is "
                     "ALU-bound, so the write rate is the conformation output rate"}


def run_long(args):
    """Long lattice chains through rosen_lattice_grow_long (hash tables of
    occupied sites in device memory), on the paper's global-memory workload:
    10^6 chains at each N.  value = nominal insertions C (N - 1) per second;
    grown = the steps the chains actually made before any dead end."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_04381_gb300 import rosen
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    Cl = args.chains or 1_000_000
    Ns = [int(v) for v in args.long_n.split(",") if v]
    parts, tot_ins, tot_ms, tot_grown, tot_lookups = {}, 0, 0.0, 0, 0
    with ClockSampler(0) as clocks:
        for Nl in Ns:
            out = rosen.lattice_outputs(Nl, Cl)
            ws = rosen.lattice_long_workspace(Nl, Cl)
            p = rosen.lattice_params(11, Nl, Cl, beta_eps=args.long_beta_eps)
            st = rosen.stats_tensor()
            rws = rosen.reduce_workspace(Cl)
            rin = rosen.lattice_reduce_in(out, Nl, use_counts=int(args.long_beta_eps == 0.0))
            for _ in range(max(1, args.warmup)):
                rosen.rosen_lattice_grow_long(p, out, ws, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                rosen.rosen_lattice_grow_long(p, out, ws, stream)
                rosen.rosen_reduce(rin, st, rws, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            grown = int(out["counts"].to(torch.int64)[:, 1:7].sum())
            sd = rosen.stats_dict(st)
            ins = Cl * (Nl - 1)
            # Expected 4x4x4-block reads per step: the end's block, plus per
            # axis the neighbouring block when the end sits on a face
            # (probability 1/2); interacting steps read it on every axis,
            # and a diagonal block when two axes sit on faces (3 x 1/4).
            lookups = 2.5 if args.long_beta_eps == 0.0 else 4.75
            parts["N%d" % Nl] = {
                "ms": ms, "insertions_per_s": ins / (ms / 1e3),
                "grown_steps_per_s": grown / (ms / 1e3), "grown_steps": grown,
                "alive_frac": sd["n_alive"] / Cl, "logZ": sd["logZ"], "mean_r2": sd["mean_r2"],
                "workspace_gb": ws.numel() * 8 / 1e9}
            tot_ins += ins
            tot_ms += ms
            tot_grown += grown
            tot_lookups += grown * lookups
            del out, ws
            torch.cuda.empty_cache()
    # Algorithmic bytes: a 16-byte entry per block read and an 8-byte bitmap
    # write per grown step.
    gbs = (tot_lookups * 16 + tot_grown * 8) / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else 0.0
    lat_ms = tot_ms
    # Real space: hard spheres, k = 32, through rosen_offlattice_grow_long.
    Cr = args.long_real_chains
    Nr = [int(v) for v in args.long_real_n.split(",") if v]
    with ClockSampler(0) as clocks_r:
        for Nl in Nr:
            out = rosen.offlattice_outputs(Nl, Cr, counters=True)
            ws = rosen.offlattice_long_workspace(Nl, Cr)
            p = rosen.offlattice_params(12, Nl, Cr, K_TRIALS)
            st = rosen.stats_tensor()
            rws = rosen.reduce_workspace(Cr)
            rin = rosen.offlattice_reduce_in(out, Nl, K_TRIALS)
            for _ in range(max(1, args.warmup)):
                rosen.rosen_offlattice_grow_long(p, out, ws, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                rosen.rosen_offlattice_grow_long(p, out, ws, stream)
                rosen.rosen_reduce(rin, st, rws, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            sd = rosen.stats_dict(st)
            ins = Cr * (Nl - 1)
            cnt = out["counters"].cpu().tolist()      # over warm-up and timed launches
            launches = max(1, args.warmup) + args.steps
            parts["hard_sphere_k32_N%d" % Nl] = {
                "ms": ms, "insertions_per_s": ins / (ms / 1e3), "chains": Cr,
                "alive_frac": sd["n_alive"] / Cr, "logZ_norm": sd["logZ_norm"],
                "mean_r2": sd["mean_r2"], "workspace_gb": ws.numel() * 8 / 1e9,
                "fp64_redecided_steps_per_chain": cnt[0] / launches / Cr}
            tot_ins += ins
            tot_ms += ms
            del out, ws
            torch.cuda.empty_cache()
    peak = measured_peak("hbm_gbs", 6800.0)
    line = {
        "metric": "long-chain insertions/s (lattice hash tables, real-space cell grids in HBM)",
        "value": tot_ins / (tot_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True,
        "dtype": "int32+fp32", "data": "synthetic",
        "config": {"workload": "lattice beta*eps %g, N in %s, %d chains each; hard spheres "
                               "k=32, N in %s, %d chains each"
                               % (args.long_beta_eps, Ns, Cl, Nr, Cr)},
        "parts": parts,
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "traffic": None,
                     "kernel": "lattice_long_kernel (lattice parts, %.1f ms)" % lat_ms,
                     "basis": "16 B per 4x4x4-block entry read (2.5 athermal, 4.75 interacting, "
                              "expected per step) + 8 B bitmap write, per grown step"},
        "clocks": clocks.summary(),
        "clocks_real_space": clocks_r.summary(),
    }
    print(json.dumps(line), flush=True)


def request_cost(e):
    """A rough relative GPU cost of a request (used only to weight a sampled
    replay): chains x N^2, real-space chains x 8k heavier than lattice ones."""
    f = 1.0 if e.model == 0 else 8.0 * e.k
    return e.C * e.N * e.N * f


def served_run(rosen, rate, duration, budget_gb, max_queue, scale, shortest_first=False,
               replay_every=0, torch=None):
    """Poisson arrivals at `rate` per second for `duration` seconds, drawn from
    the batched configuration's distribution (x scale), 20% storing their
    conformations.  After the arrivals stop, the admitted requests drain.
    Returns completed chains/s over the whole run (first arrival to last
    completion), latency percentiles and admission counts.  With
    replay_every = q, every q-th completed request (by ticket) is grown and
    reduced again, one after another, through the single-ensemble entry
    points; the single path's time for all completed requests is estimated
    from that sample (weighted by request_cost) and compared with the
    served wall time."""
    import random
    import numpy as np
    pool = batch_config(rosen, n_ens=4096, seed=5, scale=scale)
    rng = random.Random(5)
    srv = rosen.RosenServer(mem_budget_bytes=int(budget_gb * (1 << 30)), max_slots=64,
                            max_queue=max_queue, shortest_first=shortest_first)
    done, rejected, tickets, reqs = [], 0, [], {}
    lock = threading.Lock()
    stop = threading.Event()

    def collector():
        while not stop.is_set() or tickets:
            with lock:
                pending = list(tickets)
            for t in pending:
                st, res = srv.poll(t)
                if st == rosen.ROSEN_OK:
                    done.append(res)
                    srv.release(t)
                    with lock:
                        tickets.remove(t)
            time.sleep(0.005)

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    t0_ns = time.monotonic_ns()
    t_next = t0
    n = 0
    chains_offered = 0
    while True:
        t_next += rng.expovariate(rate)
        if t_next - t0 > duration:
            break
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        e = pool[n % len(pool)]
        n += 1
        req = rosen.request(e.model, e.N, e.C, e.seed + 7919 * n, e.ensemble, k=e.k,
                            potential=e.potential, beta_eps=e.beta_eps,
                            store_coords=rng.random() < 0.2)
        chains_offered += e.C
        st, t = srv.try_submit(req)
        if st == rosen.ROSEN_OK:
            with lock:
                tickets.append(t)
            reqs[t] = req
        else:
            rejected += 1
    arrivals_s = time.perf_counter() - t0
    stop.set()
    th.join(timeout=duration * 4 + 120)
    srv.close()
    ok = [r for r in done if r["status"] == rosen.ROSEN_OK]
    # The run lasts from the first arrival to the last completion (steady
    # clock of the server's time stamps).
    wall = (max(r["t_done_ns"] for r in ok) - t0_ns) / 1e9 if ok else arrivals_s
    lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in ok]) if ok else np.zeros(1)
    chains = sum(int(r["stats"]["n"]) for r in ok)
    insertions = sum(reqs[r["ticket"]].C * (reqs[r["ticket"]].N - 1) for r in ok)
    out = {"chains_per_s": chains / wall, "insertions_per_s": insertions / wall,
           "offered_requests": n, "rejected_busy": rejected, "completed": len(ok),
           "failed": len(done) - len(ok), "offered_chains_per_s": chains_offered / duration,
           "latency_ms": {"p50": float(np.percentile(lat, 50)),
                          "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
           "wall_s": wall, "arrivals_s": arrivals_s, "rate_per_s": rate,
           "duration_s": duration, "budget_gb": budget_gb, "max_queue": max_queue,
           "store_coords_fraction": 0.2, "shortest_first": bool(shortest_first)}
    if replay_every and ok:
        by_ticket = {r["ticket"]: r for r in ok}
        order = sorted(by_ticket)
        picked = order[::replay_every]
        sample = [reqs[t] for t in picked]
        ms, each = replay_single(rosen, torch, sample)
        w_all = sum(request_cost(reqs[t]) for t in order)
        w_smp = sum(request_cost(e) for e in sample)
        est = ms / 1e3 * w_all / w_smp
        # Slowdown: a sampled request's served latency over its own time on
        # an idle GPU (grow + reduce alone); latency by that time.
        alone = np.array(each)
        lat_s = np.array([(by_ticket[t]["t_done_ns"] - by_ticket[t]["t_submit_ns"]) / 1e6
                          for t in picked])
        slow = lat_s / np.maximum(alone, 1e-3)
        bins = {}
        for name, lo_ms, hi_ms in (("alone_lt_10ms", 0.0, 10.0), ("alone_10_100ms", 10.0, 100.0),
                                   ("alone_ge_100ms", 100.0, float("inf"))):
            sel = (alone >= lo_ms) & (alone < hi_ms)
            if sel.any():
                bins[name] = {"requests": int(sel.sum()),
                              "p50": float(np.percentile(lat_s[sel], 50)),
                              "p99": float(np.percentile(lat_s[sel], 99)),
                              "max": float(lat_s[sel].max())}
        out["single_path"] = {
            "replayed_requests": len(sample), "replayed_ms": ms,
            "estimated_s_for_all_completed": est,
            "served_over_single": est / wall,
            "basis": "every %d-th completed request grown and reduced alone through "
                     "rosen_*_grow + rosen_reduce, scaled to all completed requests by "
                     "C N^2 (x 8k for real space)" % replay_every}
        out["slowdown"] = {"p50": float(np.percentile(slow, 50)),
                           "p99": float(np.percentile(slow, 99)), "max": float(slow.max()),
                           "basis": "served latency / time alone, over the replayed sample"}
        out["latency_ms_by_time_alone"] = bins
        out["time_alone_ms"] = {"p50": float(np.percentile(alone, 50)),
                                "p99": float(np.percentile(alone, 99)),
                                "max": float(alone.max())}
    return out


def offered_capacity(rosen, torch, every=17):
    """Requests/s one GPU serves from the offered mix: 1 / the mean time of a
    request grown and reduced alone, over every `every`-th request of the
    arrival pool (the mix as offered, not as completed; an odd stride, since
    the pool alternates lattice and real-space requests)."""
    pool = batch_config(rosen, n_ens=4096, seed=5, scale=1.0)
    sample = pool[::every]
    ms, _ = replay_single(rosen, torch, sample)
    return 1e3 * len(sample) / ms, len(sample)


def replay_single(rosen, torch, reqs):
    """Grow and reduce the requests one after another through the
    single-ensemble entry points (CUDA events): total ms and ms per request."""
    stream = torch.cuda.current_stream()
    ws = rosen.reduce_workspace(max(r.C for r in reqs))
    st = rosen.stats_tensor()

    def one(r):
        if r.model == rosen.ROSEN_MODEL_LATTICE:
            o = rosen.lattice_outputs(r.N, r.C)
            rosen.rosen_lattice_grow(rosen.lattice_params(r.seed, r.N, r.C, beta_eps=r.beta_eps,
                                                          ensemble=r.ensemble), o, stream)
            rosen.rosen_reduce(rosen.lattice_reduce_in(o, r.N, int(r.beta_eps == 0.0)), st, ws,
                               stream)
        else:
            o = rosen.offlattice_outputs(r.N, r.C)
            rosen.rosen_offlattice_grow(
                rosen.offlattice_params(r.seed, r.N, r.C, r.k, potential=r.potential,
                                        beta_eps=r.beta_eps, ensemble=r.ensemble), o, stream)
            rosen.rosen_reduce(rosen.offlattice_reduce_in(o, r.N, r.k), st, ws, stream)
        return o

    keep = [one(r) for r in reqs[:2]]      # warm-up (allocator, modules)
    torch.cuda.synchronize()
    del keep
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    each = []
    for r in reqs:
        o = None
        e0.record(stream)
        o = one(r)
        e1.record(stream)
        torch.cuda.synchronize()
        each.append(e0.elapsed_time(e1))
        del o
    return sum(each), each


def run_served(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_04381_gb300 import rosen
    torch.cuda.set_device(0)
    r = served_run(rosen, args.rate, args.duration, args.budget_gb, args.max_queue,
                   args.batch_scale, shortest_first=args.shortest_first,
                   replay_every=args.replay_every, torch=torch)
    line = {
        "metric": "served chains/s with p50/p99 latency (Poisson arrivals)",
        "value": r["chains_per_s"], "unit": "chains/s", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "requests from the batched distribution x %g, 20%% store "
                               "conformations" % args.batch_scale, "rate_per_s": args.rate,
                   "duration_s": args.duration, "budget_gb": args.budget_gb,
                   "max_queue": args.max_queue, "shortest_first": args.shortest_first},
        "served": r,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-served", action="store_true",
                    help="step: skip the served runs (2000 requests/s, then 0.7 x capacity)")
    ap.add_argument("--no-batched", action="store_true",
                    help="step: skip the batched configuration (one graph launch)")
    ap.add_argument("--no-store-coords", action="store_true",
                    help="step: skip the hard-sphere launch that stores conformations")
    ap.add_argument("--no-perm", action="store_true", help="step: skip the PERM run")
    ap.add_argument("--served-duration", type=float, default=60.0,
                    help="step: seconds of arrivals in each served run")
    ap.add_argument("--served-policy", default="shortest_first",
                    choices=["shortest_first", "arrival"],
                    help="step: the server's scheduling policy")
    ap.add_argument("--lattice-only", action="store_true")
    ap.add_argument("--chains", type=int, default=None,
                    help="chains per ensemble (default 10^7); smaller values are for profiling")
    ap.add_argument("--workload", default="step",
                    choices=["step", "batched", "served", "long", "perm", "store"])
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="scale of the chain counts in the batched/served modes")
    ap.add_argument("--rate", type=float, default=2000.0, help="served: arrivals per second")
    ap.add_argument("--duration", type=float, default=20.0, help="served: seconds of arrivals")
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--max-queue", type=int, default=256)
    ap.add_argument("--shortest-first", action="store_true",
                    help="served: shortest remaining work first (default: arrival order)")
    ap.add_argument("--replay-every", type=int, default=0,
                    help="served: replay every q-th completed request through the single path")
    ap.add_argument("--max-attempts", type=int, default=0,
                    help="step: restart mode, growths per chain (0/1: dead ends keep W = 0)")
    ap.add_argument("--real", default="hard_sphere", choices=["hard_sphere", "lj"],
                    help="step: the real-space ensemble (default: hard spheres, k = 32)")
    ap.add_argument("--real-k", type=int, default=32)
    ap.add_argument("--real-beta-eps", type=float, default=1.0,
                    help="step: LJ well depth over kT (with --real lj)")
    ap.add_argument("--long-n", default="1000,10000", help="long: chain lengths")
    ap.add_argument("--long-beta-eps", type=float, default=0.0)
    ap.add_argument("--long-real-n", default="1000,10000", help="long: real-space lengths")
    ap.add_argument("--long-real-chains", type=int, default=100_000)
    args = ap.parse_args()
    global K_TRIALS, REAL_POT, REAL_BETA
    K_TRIALS = args.real_k
    REAL_POT = args.real
    REAL_BETA = args.real_beta_eps if args.real == "lj" else 0.0
    if args.workload == "long":
        return run_long(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "perm":
        return run_perm(args)
    if args.chains:
        global C
        C = args.chains
    if args.workload == "store":
        return run_store(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
