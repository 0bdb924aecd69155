"""Benchmark of the exchange build: K builds/s on the 64-centre diamond cell.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode f16x3|fp64]
                    [--impl xk|reference]

One step is one complete occ-RI robust-PS exchange build (orbitals, pair
kernel, the three lines, K_{mu i}, E_x) of the seeded synthetic 64-centre
cell (N=832, n=128, N_g=60^3, N_aux=4000) for the next C of a seeded
pseudo-SCF sequence.  `value` times K builds of the default tensor-core path
(--mode f16x3) on device-resident inputs with CUDA events on the launching
stream; `e2e` times the same builds through the blocking C-ABI call with
host buffers (H2D of C, D2H of K and E_x inside).  The FP64 path is timed on
the same cell beside it, and the line reports |dE_x| between the two for the
same C.  Every table is far larger than L2 (V alone is 3.5 GB in FP32), so
no flush is needed between builds.  Under torchrun each rank builds its own
C sequence on its own copy of the cell (weak scaling, no collective on the
data path); rank 0 prints one JSON line with the max-over-ranks time.

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (one full build per step) and prints the same line with
"impl": "reference".
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from cellgen import config_spec, load_cell, pseudo_scf_sequence  # noqa: E402

WORKLOAD = ("64-centre 2x2x2 diamond supercell, L=13.48 bohr, 13 Gaussians/centre "
            "(2s,2p,1d), N=832, n_occ=128, 60^3 grid, N_aux=4000")
METRIC = "K builds/s (64-atom cell)"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes per (X row, Y row) pair of the pair kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum = 1496 MB over 3.2316e8 pairs)
PAIR_DRAM_BYTES_PER_PAIR = 1496e6 / (2.0 * 1755 * 91125 + 1755.0 * 1755)
# The same for the fused role (one pass over V^T per N_aux x N_g pair): one ncu
# capture on the 27-centre cell with n = 128, 827 MB over 1.630e8 pairs
# (profiles/pair_kernel_fused_cubic27_n128.md).
FUSED_DRAM_BYTES_PER_PAIR = 827e6 / (1755.0 * 91125 + 1755.0 * 1755)
# FP64 on the CUDA cores of GB300: 2 DFMA (4 flops) per clock per SM, measured
# 3.81 flops/clock/SM with an FMA-chain probe; x 152 SMs x 2070 MHz.
FP64_FLOPS_PER_CLK_SM = 4.0
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=0)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--mode", default="f16x3", choices=["f16x3", "fp64"])
    p.add_argument("--impl", default="xk", choices=["xk", "reference"])
    p.add_argument("--config", type=int, default=2,
                   help="2: the 64-centre cell (the metric's workload); 1 or 4 for smaller cases; "
                        "3: the 216-centre cell (tables formed on the GPU, one JSON line)")
    p.add_argument("--k", type=int, default=None, help="lattice size of config 4 (k^3 centres)")
    p.add_argument("--n-occ", type=int, default=None,
                   help="override the number of occupied orbitals (profiling cases only)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    p.add_argument("--no-serve", action="store_true", help="skip the serving-latency loop")
    p.add_argument("--no-energy", action="store_true", help="skip the energy-only timing")
    p.add_argument("--no-full", action="store_true", help="skip the full K_mu_nu timing")
    p.add_argument("--isdf", action="store_true",
                   help="form the handle's ISDF tables on the GPU (xk_setup_isdf) instead of "
                        "taking the generator's, and report the set-up time")
    p.add_argument("--mix125", type=int, default=0,
                   help="run only the config-4 mix with 125-centre members: this many cells "
                        "drawn from 8/27/64/125 centres (batch and serving), one JSON line")
    p.add_argument("--batch", type=int, default=32,
                   help="cells in the grouped batch / mixed serving run (0 skips both)")
    p.add_argument("--shard", action="store_true",
                   help="under torchrun: split the interpolation points over the ranks "
                        "(xk_setup_shard) and sum K and E_x with one allreduce per build "
                        "(strong scaling) instead of one independent build per rank")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return FALLBACK_PEAKS, "fallback"


def large_pair_issued(n, Ng, Na):
    """Split MMA FLOPs issued by the n > 128 pair step: the T products (six
    piece products of K = npad), then M2 = T_A Psi, M3 = T_C Psi_g and
    M1^T = T_A^T Psi_g (four products each, N padded to 256-column tiles)."""
    npad = -(-n // 64) * 64
    nw = -(-n // 256) * 256
    return (6 * 2.0 * Na * (Ng + Na) * npad
            + 4 * 2.0 * Na * Ng * nw + 4 * 2.0 * Na * Na * nw + 4 * 2.0 * Ng * Na * nw)


def step_flops(N, n, Ng, Na):
    """Algorithmic FLOPs of each build step (the contraction counts of the
    steps listed in include/xk.h); the pair kernel counts P once."""
    return {
        "orbitals": 2.0 * Ng * N * n,
        "pair": 2.0 * Na * Ng * n + Na * Ng,
        "m2": 2.0 * Na * Ng * n,
        "m1": 2.0 * Na * Ng * n,
        "line1": 2.0 * n * Ng * N,
        "line2": 2.0 * n * Na * N,
        "line3": 4.0 * Na * Na * n + 2.0 * n * Na * N + Na * Na,
        "assemble": 4.0 * N * n,
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.proc = None
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if uuid:
                cmd += ["-i", uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cell = load_cell(config_spec(args.config, k=args.k))
    workload = WORKLOAD if args.config == 2 else (
        f"{cell.spec.name}: N={cell.N}, n={cell.n}, N_g={cell.Ng}, N_aux={cell.Naux}")
    steps = args.steps or 5
    Cs = pseudo_scf_sequence(cell.S, cell.C, steps + args.warmup, 77)
    for i in range(args.warmup):
        oracle.exx_rps_occri(cell.phi, cell.idx, cell.V, cell.W, Cs[i], cell.dV)
    t0 = time.perf_counter()
    for i in range(steps):
        oracle.exx_rps_occri(cell.phi, cell.idx, cell.V, cell.W, Cs[args.warmup + i], cell.dV)
    dt = time.perf_counter() - t0
    v = steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "builds/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded cell generator)",
        "config": {"workload": workload, "impl": "FP64 NumPy oracle of Eq. exoccri"},
        "cpu_baseline": {"value": v, "unit": "builds/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{steps} full builds of the {cell.spec.name} cell"},
        "e2e": {"value": v, "unit": "builds/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(value, dist, device):
    """The largest `value` over all ranks (the whole-job time of a step loop)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_slices(naux, world):
    """Contiguous slices [g0, g1) of the interpolation points, one per rank."""
    b = [round(r * naux / world) for r in range(world + 1)]
    return list(zip(b[:-1], b[1:]))


def reduce_partials(K, E, dist):
    """Sum the ranks' shares of K_{mu i} (N x n) and E_x (one element) in
    place with one allreduce (the only exchange of the g-sharded build)."""
    if dist is None:
        return K, E
    import torch
    buf = torch.cat([K.reshape(-1), E.reshape(-1)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    K.copy_(buf[:-1].reshape(K.shape))
    E.copy_(buf[-1:])
    return K, E


def job_throughput(world, steps, ms):
    """Whole-job builds/s: every rank runs `steps` builds; the job takes the
    slowest rank's `ms` (weak scaling, no data-path collective)."""
    return world * steps / (ms * 1e-3)


def time_device_builds(xk, h, Cd, Kd, Ed, stream, warm, steps, torch, dist=None):
    """Warm-up, then `steps` builds between CUDA events on `stream` (with
    `dist`, each build is a shard's and its share is allreduced in the step),
    as a caller runs them (the tensor path replays its captured build graph);
    then the same builds again with the per-step event timing on (which
    enqueues the kernels one by one between events) for the step times.
    Returns (ms, launches, step times)."""
    for i in range(warm):
        h.build_device(Cd[i].data_ptr(), Kd.data_ptr(), Ed.data_ptr(), stream.cuda_stream)
        reduce_partials(Kd, Ed, dist)
    torch.cuda.synchronize()
    launches0 = xk.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        h.build_device(Cd[warm + i].data_ptr(), Kd.data_ptr(), Ed.data_ptr(), stream.cuda_stream)
        reduce_partials(Kd, Ed, dist)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = xk.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    h.timing(True)
    for i in range(min(steps, 20)):
        h.build_device(Cd[warm + i].data_ptr(), Kd.data_ptr(), Ed.data_ptr(), stream.cuda_stream)
        reduce_partials(Kd, Ed, dist)
    torch.cuda.synchronize()
    st = h.step_times()
    h.timing(False)
    # the step-timed builds must leave the same K and E_x as the last timed one
    h.build_device(Cd[warm + steps - 1].data_ptr(), Kd.data_ptr(), Ed.data_ptr(), stream.cuda_stream)
    reduce_partials(Kd, Ed, dist)
    torch.cuda.synchronize()
    return ms, launches, st


def time_energy(xk, h, Cd, stream, warm, steps, torch):
    """Warm-up, then `steps` energy-only evaluations (xk_energy_device)
    between CUDA events on `stream`.  Returns (ms, step times, last E_x)."""
    Ee = torch.empty(1, dtype=torch.float64, device="cuda")
    for i in range(warm):
        h.energy_device(Cd[i].data_ptr(), Ee.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    h.timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        h.energy_device(Cd[warm + i].data_ptr(), Ee.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    st = h.step_times()
    h.timing(False)
    return e0.elapsed_time(e1), st, float(Ee.item())


def serve_latency(xk, cell, handles, Cs, rate, count, seed):
    """Serving loop: `count` build requests arrive as a Poisson process of
    `rate` per second, each from one of the SCF runs (handles) in turn, and
    are submitted with xk_submit as soon as they arrive and a slot of their
    run is free; completions are found with xk_poll.  Returns latencies
    (arrival to completion, ms) and the achieved builds/s."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
    N, n = cell.N, cell.n
    pending = []          # (arrival time, handle index, request index)
    inflight = {}         # ticket -> arrival time
    lat = []
    t0 = time.perf_counter()
    nxt = 0
    while len(lat) < count:
        now = time.perf_counter() - t0
        while nxt < count and arrivals[nxt] <= now:
            pending.append((arrivals[nxt], nxt % len(handles), nxt))
            nxt += 1
        still = []
        for arr, hi, ri in pending:
            try:
                tk = handles[hi].submit(Cs[ri % len(Cs)])
                inflight[tk] = arr
            except xk.XKError as e:
                if e.code != xk.XK_EBUSY:
                    raise
                still.append((arr, hi, ri))
        pending = still
        for tk in list(inflight):
            st, _, _, _ = xk.poll(tk, N, n)
            if st == xk.XK_OK:
                lat.append(1e3 * (time.perf_counter() - t0 - inflight.pop(tk)))
        if not inflight and not pending and nxt < count:
            time.sleep(max(0.0, min(0.001, arrivals[nxt] - (time.perf_counter() - t0))))
    total = time.perf_counter() - t0
    return np.array(lat), count / total


def serve_mix(xk, handles, seqs, rate, count, seed):
    """Serving over runs of different cell sizes: `count` requests arrive as
    a Poisson process of `rate` per second from the runs in turn (run r's
    requests walk its own pseudo-SCF sequence), are submitted as soon as a
    slot of their run is free and collected with xk_poll.  Returns the
    latencies (ms) and the achieved builds/s."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
    pending, inflight, lat = [], {}, []
    t0 = time.perf_counter()
    nxt = 0
    while len(lat) < count:
        now = time.perf_counter() - t0
        while nxt < count and arrivals[nxt] <= now:
            pending.append((arrivals[nxt], nxt % len(handles), nxt // len(handles)))
            nxt += 1
        still = []
        for arr, r, k in pending:
            try:
                tk = handles[r].submit(seqs[r][k % len(seqs[r])])
                inflight[tk] = (arr, r)
            except xk.XKError as e:
                if e.code != xk.XK_EBUSY:
                    raise
                still.append((arr, r, k))
        pending = still
        for tk in list(inflight):
            arr, r = inflight[tk]
            st, _, _, _ = xk.poll(tk, handles[r].N, handles[r].n)
            if st == xk.XK_OK:
                lat.append(1e3 * (time.perf_counter() - t0 - arr))
                del inflight[tk]
        if not inflight and not pending and nxt < count:
            time.sleep(max(0.0, min(0.001, arrivals[nxt] - (time.perf_counter() - t0))))
    return np.array(lat), count / (time.perf_counter() - t0)


def batch_and_mixed_serving(xk, cell64, count, seed=4000):
    """Config-4 and config-5 shaped runs on one GPU: `count` cells drawn with
    the seed from {8, 27, 64} centres (n = 2 per centre, N_aux = 5 N for the
    cubic cells; the 64-centre member is the benchmark cell), each a handle
    with its own tables and pseudo-SCF coefficients.  (a) one build of every
    cell as one xk_batch (CUDA graph, grouped pair launches) against the same
    builds one xk_build at a time; (b) serving: Poisson arrivals from all
    runs at 0.25, 0.5 and 1.0 x the one-at-a-time throughput."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([8, 27, 64], size=count)
    cells = {8: load_cell(config_spec(4, k=2)), 27: load_cell(config_spec(4, k=3)), 64: cell64}
    return batch_and_serve(xk, cells, sizes)


def batch_and_serve(xk, cells, sizes):
    """(a) and (b) of batch_and_mixed_serving over the given cells (size ->
    cell) and member sizes."""
    count = len(sizes)
    handles, seqs = [], []
    for i, z in enumerate(sizes):
        c = cells[int(z)]
        handles.append(xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3"))
        seqs.append(pseudo_scf_sequence(c.S, c.C, 8, 5000 + i))
    footprint = sum(xk.footprint(h.Ng, h.N, h.n, h.Naux, "f16x3") for h in handles)
    out = {"cells": int(count), "sizes": {str(z): int(np.sum(sizes == z)) for z in sorted(cells)},
           "device_bytes": int(footprint)}
    try:
        b = xk.Batch(handles)
        try:
            first = [q[0] for q in seqs]
            b.build(first)  # captures the graph
            b.build(first)
            reps = 4
            t0 = time.perf_counter()
            for r in range(reps):
                b.build([q[1 + r] for q in seqs])
            tb = (time.perf_counter() - t0) / reps
        finally:
            b.release()
        t0 = time.perf_counter()
        for r in range(2):
            for h, q in zip(handles, seqs):
                h.build(q[5 + r])
        ts = (time.perf_counter() - t0) / 2
        out["batch"] = {"builds_per_s": count / tb, "ms_per_batch": 1e3 * tb,
                        "one_at_a_time_builds_per_s": count / ts,
                        "note": "host C in, host K and E_x out; one CUDA graph per batch with "
                                "the pair contractions of all members in grouped launches"}
        cap = count / ts
        rates = []
        for frac in (0.25, 0.5, 1.0):
            lat, got = serve_mix(xk, handles, seqs, frac * cap, 2 * count if frac < 1 else 3 * count, 11)
            rates.append({"arrival_rate_per_s": frac * cap, "requests": int(lat.size),
                          "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)), "builds_per_s": got})
        out["serving"] = {"runs": int(count), "rates": rates,
                          "note": "xk_submit/xk_poll, four slots per run, runs of " +
                                  ", ".join(str(z) for z in sorted(cells)) +
                                  " centres overlapping on the GPU"}
    finally:
        for h in handles:
            h.release()
    return out


def scf_runs_queued(xk, cell64, count=48, builds=6, seed=4800, budget_runs=12):
    """Config-5 shaped serving with queued admission: `count` SCF runs drawn
    with the seed from {8, 27, 64} centres arrive as a Poisson process; each
    run is admitted by xk_setup_queued against an HBM budget that holds about
    `budget_runs` runs of the mix (XK_HBM_BUDGET_BYTES over what is already
    admitted), does `builds` builds of its own pseudo-SCF sequence (xk_build,
    one thread per run, so builds of different runs overlap on the device) and
    releases its tables, which admits the next waiting run.
    Arrival rates 0.25, 0.5 and 1.0 x the budget's capacity (budget_runs
    64-centre runs live at a time, each as long as one alone takes).  Reports
    admission waits and build latencies (request to K on the host)."""
    import threading
    rng = np.random.default_rng(seed)
    sizes = rng.choice([8, 27, 64], size=count)
    cells = {8: load_cell(config_spec(4, k=2)), 27: load_cell(config_spec(4, k=3)), 64: cell64}
    seqs = [pseudo_scf_sequence(cells[int(z)].S, cells[int(z)].C, builds, 6000 + i)
            for i, z in enumerate(sizes)]
    fp = {z: xk.footprint(c.Ng, c.N, c.n, c.Naux, "f16x3") for z, c in cells.items()}
    mean_fp = float(np.mean([fp[int(z)] for z in sizes]))
    # one 64-centre run alone (set-up, builds, release): the capacity of the
    # budget is budget_runs such runs live at a time
    c = cells[64]
    t0 = time.perf_counter()
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    for k in range(builds):
        h.build(c.C)
    h.release()
    run_s = time.perf_counter() - t0
    setup_alone = {}
    for z, cz in cells.items():  # one set-up of each size with nothing else running
        t1 = time.perf_counter()
        hz = xk.Handle(cz.phi, cz.idx, cz.V, cz.W, cz.dV, cz.n, mode="f16x3")
        setup_alone[str(z)] = time.perf_counter() - t1
        hz.release()
    base, _ = xk.admit_state()
    budget = int(budget_runs * mean_fp)
    sustain = budget_runs / run_s  # runs/s at which the budget is full on average
    old = os.environ.get("XK_HBM_BUDGET_BYTES")
    os.environ["XK_HBM_BUDGET_BYTES"] = str(base + budget)
    out = {"runs": int(count), "sizes": {str(z): int(np.sum(sizes == z)) for z in (8, 27, 64)},
           "builds_per_run": builds, "budget_bytes": budget, "run_alone_s_64": run_s,
           "setup_alone_s": setup_alone,
           "budget_in_runs_of_the_mix": budget_runs, "rates": []}
    try:
        for frac in (0.25, 0.5, 1.0):
            rate = frac * sustain
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
            waits, lats, errs = [], [], []
            lock = threading.Lock()
            t_start = time.perf_counter()

            def run(i):
                z = int(sizes[i])
                cc = cells[z]
                delay = arrivals[i] - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
                ta = time.perf_counter()
                try:
                    hh = xk.Handle(cc.phi, cc.idx, cc.V, cc.W, cc.dV, cc.n, mode="f16x3",
                                   queue_timeout_ms=120000.0)
                except xk.XKError as e:
                    with lock:
                        errs.append(str(e))
                    return
                tw = time.perf_counter() - ta
                my = []
                try:
                    for k in range(builds):
                        tr = time.perf_counter()
                        hh.build(seqs[i][k])
                        my.append(1e3 * (time.perf_counter() - tr))
                finally:
                    hh.release()
                with lock:
                    waits.append(1e3 * tw)
                    lats.extend(my)

            ths = [threading.Thread(target=run, args=(i,)) for i in range(count)]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
            total = time.perf_counter() - t_start
            lats = np.array(lats)
            waits = np.array(waits)
            out["rates"].append({
                "run_arrival_rate_per_s": rate, "x_sustained": frac,
                "admission_wait_ms": {"p50": float(np.percentile(waits, 50)),
                                      "p99": float(np.percentile(waits, 99)),
                                      "max": float(waits.max())} if waits.size else None,
                "build_latency_ms": {"p50": float(np.percentile(lats, 50)),
                                     "p99": float(np.percentile(lats, 99))} if lats.size else None,
                "builds_per_s": float(lats.size / total), "seconds": total,
                "errors": errs[:3]})
    finally:
        if old is None:
            del os.environ["XK_HBM_BUDGET_BYTES"]
        else:
            os.environ["XK_HBM_BUDGET_BYTES"] = old
    out["note"] = ("xk_setup_queued admission (arrival order, woken by xk_release), one thread "
                   "per run doing blocking xk_build calls; admission_wait_ms is the whole "
                   "xk_setup_queued call: the wait in the queue plus the set-up itself (the "
                   "upload and conversion of the run's tables from pageable host memory, shared "
                   "by the set-ups that run at the same time); 125- and 216-centre members left "
                   "out (host generation of their tables takes minutes)")
    return out


def run_mix125(args):
    """The grouped batch with its largest cell size: `args.mix125` cells drawn with seed 4125
    from {8, 27, 64, 125} centres.  The 125-centre cell (N = 1625, n = 250,
    75^3 grid, N_aux = 8125) gets its ISDF tables on the GPU (xk_setup_isdf,
    FP64; the host fit would take hours), read back and handed to its f16x3
    members like any caller's tables.  Then the grouped batch against one
    build at a time, and serving at three rates (batch_and_serve).  32 cells
    drawn the same way would need the footprint reported as
    `footprint_of_32_cells`, more than one GPU holds."""
    import dataclasses
    import torch
    import paper_2207_04636_gb300 as xk
    from paper_2207_04636_gb300 import build as xkbuild
    from cellgen import build_cell
    xkbuild.build_library()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    c125 = build_cell(config_spec(4, k=5), fit=False)
    t_inputs = time.perf_counter() - t0
    t0 = time.perf_counter()
    hf = xk.Handle.isdf(c125.phi, c125.idx, c125.grid, c125.L, c125.n, mode="fp64")
    t_isdf = time.perf_counter() - t0
    W, V, ridge = hf.tables(np.arange(c125.Naux))
    hf.release()
    c125 = dataclasses.replace(c125, V=V, W=W)
    cells = {8: load_cell(config_spec(4, k=2)), 27: load_cell(config_spec(4, k=3)),
             64: load_cell(config_spec(2)), 125: c125}
    fp = {z: xk.footprint(c.Ng, c.N, c.n, c.Naux, "f16x3") for z, c in cells.items()}
    rng = np.random.default_rng(4125)
    sizes = rng.choice([8, 27, 64, 125], size=args.mix125)
    fp32 = sum(fp[int(z)] for z in np.random.default_rng(4125).choice([8, 27, 64, 125], size=32))
    res = batch_and_serve(xk, cells, sizes)
    line = {"metric": "K builds/s (grouped batch of 8- to 125-centre cells)",
            "value": res.get("batch", {}).get("builds_per_s"), "unit": "builds/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f16x3",
            "data": "synthetic (seeded cell generator; 125-centre ISDF tables formed on the GPU)",
            "config": {"workload": f"{args.mix125} cells drawn from 8/27/64/125 centres (seed 4125)"},
            "footprint_bytes": {str(z): int(v) for z, v in fp.items()},
            "footprint_of_32_cells": int(fp32),
            "device_memory_bytes": int(torch.cuda.get_device_properties(0).total_memory),
            "setup_125_s": {"host_inputs": t_inputs, "isdf_fp64_on_gpu": t_isdf},
            "isdf_ridge_125": ridge, "mix": res}
    print(json.dumps(line), flush=True)


def gpu_points(xk, cell):
    """The two-stage point selection of Sec. IV.C with the pivoting on the GPU
    (xk_isdf_points): per-atom candidates from each Voronoi cell of the grid,
    then a global pivoting over their union.  Returns (sorted idx, seconds)."""
    t0 = time.perf_counter()
    x = np.arange(cell.grid) * (cell.L / cell.grid)
    pts = np.stack(np.meshgrid(x, x, x, indexing="ij"), axis=-1).reshape(-1, 3)
    owner = np.zeros(pts.shape[0], dtype=np.int64)
    best = np.full(pts.shape[0], np.inf)
    for i, a in enumerate(cell.centres):
        d = pts - a
        d -= cell.L * np.round(d / cell.L)
        r2 = np.einsum("ij,ij->i", d, d)
        m = r2 < best
        best[m] = r2[m]
        owner[m] = i
    per_atom = int(np.ceil(cell.Naux / cell.N * (cell.N // len(cell.centres)))) + 10
    cand = []
    for i in range(len(cell.centres)):
        loc = np.nonzero(owner == i)[0]
        cand.append(loc[xk.isdf_points(cell.phi[loc], per_atom)])
    cand = np.unique(np.concatenate(cand))
    idx = np.sort(cand[xk.isdf_points(cell.phi[cand], cell.Naux)])
    return idx, time.perf_counter() - t0


def run_config3(args):
    """The 216-centre cell (N = 2808, n = 432, 90^3 grid, N_aux = 13500): its
    ISDF tables are formed on the GPU (xk_setup_isdf, FP64) because the host
    fit takes hours.  Sequence: the FP64 handle's set-up and one FP64 build;
    its V and W read back to the host (79 GB); the handle released; the
    tensor-path handle set up from those tables; timed builds; the closed-form
    E_x of the oracle on the host from the same tables (parity at full size)."""
    import torch
    import oracle
    import paper_2207_04636_gb300 as xk
    from paper_2207_04636_gb300 import build as xkbuild
    from cellgen import build_cell
    xkbuild.build_library()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    cell = build_cell(config_spec(3), fit=False)
    t_inputs = time.perf_counter() - t0
    N, n, Ng, Na = cell.N, cell.n, cell.Ng, cell.Naux
    steps = args.steps or 10
    warm = max(3, args.warmup)
    Cs = pseudo_scf_sequence(cell.S, cell.C, steps + warm, 3000)
    C_last = Cs[-1]
    t0 = time.perf_counter()
    hf = xk.Handle.isdf(cell.phi, cell.idx, cell.grid, cell.L, n, mode="fp64")
    t_isdf = time.perf_counter() - t0
    t0 = time.perf_counter()
    K64, E64 = hf.build(C_last)
    t_fp64 = time.perf_counter() - t0
    W, V, ridge = hf.tables(np.arange(Na))
    hf.release()
    t0 = time.perf_counter()
    h = xk.Handle(cell.phi, cell.idx, V, W, cell.dV, n, mode="f16x3")
    t_mixed_setup = time.perf_counter() - t0
    Cd = [torch.from_numpy(C).cuda() for C in Cs]
    Kd = torch.empty((N, n), dtype=torch.float64, device="cuda")
    Ed = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(None)
    ms, launches, st = time_device_builds(xk, h, Cd, Kd, Ed, stream, warm, steps, torch)
    clocks = sampler.stop()
    K, E = Kd.cpu().numpy(), float(Ed.item())
    tuned = h.autotune_info()
    h.release()
    line = {"metric": "K builds/s (216-centre cell)", "value": steps / (ms * 1e-3),
            "unit": "builds/s", "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": ms / steps, "higher_is_better": True, "dtype": "f16x3",
            "data": "synthetic (seeded cell generator; ISDF tables formed on the GPU)",
            "config": {"workload": "216-centre 3x3x3 diamond supercell, L=20.22 bohr, N=2808, "
                                   "n_occ=432, 90^3 grid, N_aux=13500", "N": N, "n": n,
                       "N_g": Ng, "N_aux": Na},
            "step_ms": {k: v[0] / max(1, v[1]) for k, v in st.items() if v[1]},
            "gpu_launches": int(launches), "clocks": clocks, "autotune": tuned,
            "setup_s": {"host_inputs": t_inputs, "isdf_fp64_on_gpu": t_isdf,
                        "tensor_handle_from_tables": t_mixed_setup},
            "isdf_ridge": ridge,
            "fp64_path": {"s_per_build": t_fp64, "dE_x_vs_fp64": abs(E - E64),
                          "max_dK_vs_fp64": float(np.max(np.abs(K - K64))), "E_x_fp64": E64},
            "E_x": E}
    pk, pk_src = peaks()
    pair_ms = st["pair"][0] / max(1, st["pair"][1])
    issued = large_pair_issued(n, Ng, Na)
    line["pair_roofline"] = {
        "bound": "tensor", "pair_ms": pair_ms,
        "issued_tensor_tflops": issued / (pair_ms * 1e-3) / 1e12,
        "issued_frac": issued / (pair_ms * 1e-3) / 1e12 / pk.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]),
        "algorithmic_tflops": 6.0 * Na * Ng * n / (pair_ms * 1e-3) / 1e12,
        "peak_source": f"dense bf16/fp16 tensor rate ({pk_src})"}
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        E0 = oracle.exx_energy_direct(cell.phi, cell.idx, V, W, C_last, cell.dV)
        line["parity_oracle_closed_form"] = {
            "E_x_oracle": E0, "dE_x_fp64_path": abs(E64 - E0), "dE_x_tensor_path": abs(E - E0),
            "oracle_s": time.perf_counter() - t0,
            "note": "oracle E_x from the closed form -dV(2 sum V P^2 - sum W Q^2) on the host, "
                    "same tables and C as the last build"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == 3:
        run_config3(args)
        return
    if args.mix125:
        run_mix125(args)
        return
    import torch
    import paper_2207_04636_gb300 as xk
    from paper_2207_04636_gb300 import build as xkbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    xkbuild.build_library()

    mode = args.mode
    steps = args.steps or (200 if mode != "fp64" else 6)
    warm = max(3, args.warmup)
    spec = config_spec(args.config, k=args.k)
    if args.n_occ:
        spec.n_occ = args.n_occ
    cell = load_cell(spec)
    N, n, Ng, Na = cell.N, cell.n, cell.Ng, cell.Naux
    workload = WORKLOAD if args.config == 2 else f"{cell.spec.name}: N={N}, n={n}, N_g={Ng}, N_aux={Na}"
    shard = args.shard and world > 1
    # a sharded run builds one C sequence across all ranks; otherwise each rank its own
    Cs = pseudo_scf_sequence(cell.S, cell.C, steps + warm, 1000 + (0 if shard else rank))
    Cd = [torch.from_numpy(C).cuda() for C in Cs]
    Kd = torch.empty((N, n), dtype=torch.float64, device="cuda")
    Ed = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    t_setup = time.perf_counter()
    points = None
    if args.isdf:
        idx_gpu, t_pts = gpu_points(xk, cell)
        points = {"s": t_pts, "count": int(idx_gpu.size),
                  "same_as_generator": bool(np.array_equal(idx_gpu, np.sort(cell.idx))),
                  "common_with_generator": int(np.intersect1d(idx_gpu, cell.idx).size)}
        t_setup = time.perf_counter()
        h = xk.Handle.isdf(cell.phi, cell.idx, cell.grid, cell.L, n, mode=mode)
    elif shard:  # this rank's slice of the interpolation points
        g0, g1 = shard_slices(Na, world)[rank]
        h = xk.Handle.shard(cell.phi, cell.idx, cell.V[g0:g1], cell.W[g0:g1], g0, g1, cell.dV, n,
                            mode=mode)
    else:
        h = xk.Handle(cell.phi, cell.idx, cell.V, cell.W, cell.dV, n, mode=mode)
    t_setup = time.perf_counter() - t_setup
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    ms, launches, st = time_device_builds(xk, h, Cd, Kd, Ed, stream, warm, steps, torch,
                                          dist if shard else None)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    K_last = Kd.cpu().numpy()
    E_last = float(Ed.item())
    C_last = Cs[warm + steps - 1]
    # per-build a-posteriori estimate |E_x - E_K| (E_K = -sum K o C of the
    # returned K) of the last timed build; a shard's is its share's
    err_est = h.error_estimate()
    tuned = h.autotune_info() if mode != "fp64" else None

    # e2e through the blocking C-ABI call: host (pinned) buffers in and out
    Ch = [torch.from_numpy(C).pin_memory() for C in Cs[warm:warm + steps]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        Kh, Eh = h.build(Ch[i].numpy())
        if shard:  # the shares, summed over the ranks and read back
            Kt = torch.from_numpy(Kh).cuda()
            Et = torch.tensor([Eh], dtype=torch.float64, device="cuda")
            reduce_partials(Kt, Et, dist)
            Kh, Eh = Kt.cpu().numpy(), float(Et.item())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    energy = None
    if not args.no_energy and world == 1:
        ms_e, st_e, E_e = time_energy(xk, h, Cd, stream, warm, steps, torch)
        pair_ms = st_e["pair"][0] / max(1, st_e["pair"][1])
        npad = -(-n // 64) * 64
        # algorithmic DRAM bytes of the energy pair step: V' and W' in FP32 read
        # once, the orbital pieces (m, h) on the grid and at the points
        ebytes = 4.0 * Na * Ng + 4.0 * Na * Na + 4.0 * (Ng + Na) * npad
        pk_e, pk_src_e = peaks()
        hbm = pk_e.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
        energy = {"evals_per_s": steps / (ms_e * 1e-3), "ms_per_eval": ms_e / steps,
                  "step_ms": {k: v[0] / max(1, v[1]) for k, v in st_e.items() if v[1] > 0},
                  "E_x_last": E_e, "equals_build_E_x": E_e == E_last,
                  "roofline": {"bound": "hbm", "kernel": "energy-only pair kernel (roles A, C)",
                               "achieved": ebytes / (pair_ms * 1e-3) / 1e9, "peak": hbm,
                               "unit": "GB/s", "frac": ebytes / (pair_ms * 1e-3) / 1e9 / hbm,
                               "peak_source": f"HBM copy bandwidth ({pk_src_e})",
                               "traffic": None},
                  "note": "xk_energy_device: E_x alone from the closed form (no K), same "
                          "coefficient sequence as the builds"}
    full = None
    if not args.no_full and world == 1:
        Kf = h.build_full(C_last)  # the first call allocates the full-K scratch
        reps = 5 if mode != "fp64" else 1
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            Kf = h.build_full(C_last)
        ms_full = (time.perf_counter() - t0) * 1e3 / reps
        npad = -(-n // 64) * 64
        # algorithmic flops: S and W o Q products, M_A = T_A Phi, M_C = T_C Phi_g, Phi_g^T M (x2)
        fl_full = (2.0 * Na * Ng * n + 2.0 * Na * Na * n + 2.0 * Na * Ng * N + 2.0 * Na * Na * N
                   + 4.0 * N * N * Na)
        # split MMA work issued on the tensor path (4 passes each; S with 6 for n > 128)
        fl_issued = ((6 if n > 128 else 4) * 2.0 * Na * (Ng + Na) * npad
                     + 4 * (2.0 * Na * Ng * N + 2.0 * Na * Na * N + 4.0 * N * N * Na))
        full = {"ms_per_build": ms_full,
                "algorithmic_tflops_per_s": fl_full / (ms_full * 1e-3) / 1e12,
                "issued_tensor_tflops_per_s": fl_issued / (ms_full * 1e-3) / 1e12,
                "note": "xk_build_full: K_mu_nu (N x N) of Eq. rpsEx with the three robust-PS "
                        "terms, host buffers in and out, same C as the last build",
                "symmetry_rel": float(np.max(np.abs(Kf - Kf.T)) / np.max(np.abs(Kf))),
                "max_dKC_vs_build": float(np.max(np.abs(Kf @ C_last - K_last)))}
    h.release()
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")

    serving = None
    if mode != "fp64" and not args.no_serve and world == 1:
        runs = [xk.Handle(cell.phi, cell.idx, cell.V, cell.W, cell.dV, n, mode=mode)
                for _ in range(2)]
        rate = 0.7 * steps / (ms * 1e-3)
        lat, got = serve_latency(xk, cell, runs, Cs[warm:], rate, 400, 7)
        for r in runs:
            r.release()
        serving = {"runs": len(runs), "requests": int(lat.size), "arrival_rate_per_s": rate,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "builds_per_s": got,
                   "note": "Poisson arrivals at 0.7x the measured throughput, xk_submit/xk_poll, "
                           "host buffers in and out"}

    mixed = None
    if mode != "fp64" and args.batch > 0 and world == 1:
        mixed = batch_and_mixed_serving(xk, cell, args.batch)
        if not args.no_serve:
            mixed["scf_runs_queued"] = scf_runs_queued(xk, cell)

    fp64 = None
    if mode != "fp64" and not args.no_fp64:
        hf = xk.Handle(cell.phi, cell.idx, cell.V, cell.W, cell.dV, n, mode="fp64")
        nf = min(5, len(Cd) - 1)  # FP64 builds timed after one warm-up
        ms64, _, _ = time_device_builds(xk, hf, Cd[len(Cd) - nf - 1:], Kd, Ed, stream, 1, nf, torch)
        hf.build_device(Cd[warm + steps - 1].data_ptr(), Kd.data_ptr(), Ed.data_ptr(),
                        stream.cuda_stream)
        torch.cuda.synchronize()
        K64, E64 = Kd.cpu().numpy(), float(Ed.item())
        coul = None
        if not args.no_full:
            hf.coulomb(C_last, cell.grid, cell.L)  # the first call allocates its scratch
            t0 = time.perf_counter()
            J, EJ = hf.coulomb(C_last, cell.grid, cell.L)
            ms_j = (time.perf_counter() - t0) * 1e3
            fl_j = 2.0 * N * N * Ng + 2.0 * Ng * N * n
            coul = {"ms_per_build": ms_j, "E_J": EJ,
                    "fp64_tflops_per_s": fl_j / (ms_j * 1e-3) / 1e12,
                    "fp64_peak_tflops": FP64_FLOPS_PER_CLK_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12,
                    "note": "xk_coulomb on the FP64 handle: density, DFT Poisson solve, "
                            "J = dV Phi^T diag(v) Phi, host buffers in and out"}
        if full is not None:
            t0 = time.perf_counter()
            Kf64 = hf.build_full(C_last)
            full["fp64_path_ms"] = (time.perf_counter() - t0) * 1e3
            full["max_dK_vs_fp64"] = float(np.max(np.abs(Kf - Kf64)))
            full["max_abs_K"] = float(np.max(np.abs(Kf64)))
        hf.release()
        fp64 = {"builds_per_s": nf / (ms64 * 1e-3), "ms_per_build": ms64 / nf, "builds_timed": nf,
                "dE_x_vs_fp64": abs(E_last - E64),
                "max_dK_vs_fp64": float(np.max(np.abs(K_last - K64))), "coulomb_j": coul}

    if rank == 0:
        pk, pk_src = peaks()
        fl = step_flops(N, n, Ng, Na)
        if mode == "fp64":
            dom = max((k for k in st if st[k][1] > 0), key=lambda k: st[k][0])
            dom_ms = st[dom][0] / max(1, st[dom][1])
            peak = FP64_FLOPS_PER_CLK_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
            roof = {"bound": "alu", "kernel": f"step '{dom}' (FP64 DFMA GEMM)",
                    "achieved": fl[dom] / (dom_ms * 1e-3) / 1e12, "peak": peak,
                    "unit": "TFLOP/s",
                    "peak_source": "FP64 DFMA rate: 4 flop/clk/SM x 152 SMs x 2070 MHz",
                    "traffic": None}
        else:
            dom = "pair"
            dom_ms = st[dom][0] / max(1, st[dom][1])
            algo = fl["pair"] + fl["m2"] + fl["m1"] + 4.0 * Na * Na * n
            npad = -(-n // 64) * 64
            if npad == 128:
                # fused role: S once (4 split MMA passes) and both back-contractions
                # (3 passes each) per N_aux x N_g pair; role C: S + one product
                issued = 10 * 2.0 * Na * Ng * npad + 7 * 2.0 * Na * Na * npad
                kname = ("pair kernel (fused role: S = Psi Psi_g^T once, V^T o S, M1 and M2 "
                         "from one pass over V; role C in the same launch)")
            elif n > 128:
                issued = large_pair_issued(n, Ng, Na)
                kname = ("pair step (n > 128): T products (tprod_kernel) and the three "
                         "back-contractions on 128 x 256 tiles (gemm_wide_kernel)")
            else:
                # roles A and B each form S (4 passes) and one product (3 passes)
                issued = 7 * 2.0 * 2 * Na * Ng * npad + 7 * 2.0 * Na * Na * npad
                kname = ("pair kernel (fused P, V o P, back-contraction; roles A, B, C "
                         "in one launch per build)")
            peak = pk.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
            pair_bytes = (FUSED_DRAM_BYTES_PER_PAIR if npad == 128 else PAIR_DRAM_BYTES_PER_PAIR)
            roof = {"bound": "tensor",
                    "kernel": kname,
                    "achieved": algo / (dom_ms * 1e-3) / 1e12, "peak": peak,
                    "unit": "TFLOP/s",
                    "peak_source": f"dense bf16/fp16 tensor rate ({pk_src})",
                    "issued_tensor_tflops": issued / (dom_ms * 1e-3) / 1e12,
                    # tensor-pipe fraction: split MMA FLOPs issued over the same peak;
                    # the algorithmic 'frac' counts each product once
                    "issued_frac": issued / (dom_ms * 1e-3) / 1e12 / peak,
                    "issued_frac_of_sustained": issued / (dom_ms * 1e-3) / 1e12 / pk.get(
                        "bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]),
                    # DRAM bytes of the pair launch: dram__bytes_read + write of one ncu
                    # capture of the same kernel on the 27-centre cell with n = 128,
                    # scaled to this cell by its pair count (the traffic is per pair)
                    "traffic": (pair_bytes * (Na * Ng * (1.0 if npad == 128 else 2.0)
                                              + float(Na) * Na) if n <= 128 else None),
                    "traffic_source": ("ncu capture of the pair kernel on the 27-centre cell "
                                       "(n = 128), scaled by pair count" if n <= 128 else
                                       "not captured for this n")}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["ms_per_build"] = dom_ms
        # a sharded job completes one build per step across all ranks (strong
        # scaling); replicas complete one build per rank per step (weak scaling)
        value = job_throughput(1 if shard else world, steps, ms)
        line = {
            "metric": METRIC, "value": value, "unit": "builds/s", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "strong" if shard else "weak",
            "vs_baseline": None,
            "dtype": "f64" if mode == "fp64" else "f16x3",
            "data": "synthetic (seeded cell generator; inputs resident in HBM)"
                    + ("; ISDF tables formed on the GPU" if args.isdf else ""),
            "config": {"workload": workload, "mode": mode, "N": N, "n": n, "N_g": Ng,
                       "N_aux": Na, "l2": "inputs larger than L2 (V is N_aux x N_g)",
                       "parallelism": (f"g-sharded x{world} (one allreduce of K and E_x "
                                       "per build)" if shard else f"replicas x{world}")},
            "E_x": E_last,
            "step_ms": {k: v[0] / max(1, v[1]) for k, v in st.items()},
            "algorithmic_tflops_per_s": sum(fl.values()) / (ms * 1e-3 / steps) / 1e12,
            "roofline": roof,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "error_estimate": {"last_build": err_est,
                               "definition": "|E_x - E_K|, E_K = -sum K o C of the returned K "
                                             "(xk_poll err_est / xk_error_estimate)"},
            "autotune": tuned,
            "e2e": {"value": job_throughput(1 if shard else world, steps, e2e_s * 1e3),
                    "unit": "builds/s",
                    "h2d_bytes_per_step": N * n * 8, "d2h_bytes_per_step": N * n * 8 + 8},
        }
        if args.isdf:
            fl_isdf = (2.0 * Na * Ng * N + 2.0 * Na * Na * N + 2.0 * Na ** 3 / 3.0
                       + 2.0 * Na * Na * Ng + 2.0 * Na * Na * Ng)
            line["isdf_points_gpu"] = points
            line["isdf_setup"] = {"s": t_setup, "fp64_tflops_per_s_lower_bound":
                                  fl_isdf / t_setup / 1e12,
                                  "note": "xk_setup_isdf: X_gR, X_gg, Cholesky, chi, V, W in FP64 "
                                          "plus the handle's own set-up (the rate counts the "
                                          "ISDF products only, so it is a lower bound)"}
        if energy:
            line["energy_only"] = energy
        if full:
            line["full_k"] = full
        if fp64 and fp64.get("coulomb_j"):
            line["coulomb_j"] = fp64.pop("coulomb_j")
        if serving:
            line["serving"] = serving
        if mixed:
            line["mixed_cells"] = mixed
        if fp64:
            line["fp64_path"] = fp64
            line["speedup_vs_fp64_path"] = value / world / fp64["builds_per_s"]
        if not args.no_cpu_baseline and world == 1:
            import oracle
            t0 = time.perf_counter()
            nb = 0
            while True:
                K0, E0 = oracle.exx_rps_occri(cell.phi, cell.idx, cell.V, cell.W, C_last, cell.dV)
                nb += 1
                if time.perf_counter() - t0 > 10.0 or nb >= 3:
                    break
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": nb / dt, "unit": "builds/s", "cores": cpu_cores(),
                                    "kind": "oracle",
                                    "sample": f"{nb} full FP64 oracle builds of the same cell"}
            line["parity_last_step"] = {"dE_x_vs_oracle": abs(E_last - E0),
                                        "max_dK_vs_oracle": float(np.max(np.abs(K_last - K0)))}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
