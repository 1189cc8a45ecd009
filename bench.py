"""Benchmark of the incremental state-vector hot path (qTask, arXiv 2210.01076).

Workload (one GPU): n = 24 qubits, complex128 amplitudes (float-float
arithmetic, QT_C128_DF), 1000 random gates (~40 % multi-qubit) in ASAP levels,
partitions of 2^16 amplitudes, a checkpoint every 8 levels.  A *step* is one
incremental round: 1-5 random edits (insert / remove / replace at uniformly
random levels) followed by qt_update_state -- every row of the hot path
(circuit store, planning and fusion, dirty tracking, checkpoint restart, the
gate kernels).  The state (256 MiB) is larger than L2, so no flush is needed.

Metric: amplitude-updates/s (sum over gates of the amplitudes each gate's
pass processed, per second of device time), with HBM GB/s, the per-round
latency p50/p99 against a full re-simulation, and the clean fraction.

``--impl reference`` times the FP64 CPU oracle (the only reference: the paper
ships no code) on the same workload, one bounded sample per step.
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

N_QUBITS = 24
N_GATES = 1000
LOG2_PART = 16
CKPT = 8  # levels per checkpoint segment: the measured best p50 round latency (4..24 swept)
P_MULTI = 0.4
SEED = 2210
WORKLOAD = "incremental random circuit n=24, 1000 gates (~40% multi-qubit), 1-5 edits/round, partitions 2^16"


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def rank_seed(rank: int) -> int:
    """Each rank simulates its own circuit (independent replicas: weak scaling)."""
    return SEED + 1000 * rank


def aggregate_over_ranks(units: float, seconds: float, device=None):
    """Whole-job (units, seconds) over all ranks: the units every rank
    processed, summed, and the slowest rank's time, which bounds the job.
    One rank (or no process group): returned unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(seconds)
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    a = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(a)
    return float(a.item()), float(t.item())


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("qt_kernels.cu", "qt_pass_reg.cu", "qt_arith.cuh", "qt_internal.h", "qt_tc.cuh", "qt_launch.cuh"):
        with open(os.path.join(ROOT, "paper_2210_01076_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_hash, name="k_pass_df_traffic.json"):
    """DRAM bytes per amplitude-pass of the fused-pass kernel from a committed
    ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") == kernel_hash:
            return d
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


# The paper's own results, quoted for context only: they are CPU wall-clock
# ratios of its simulator over two others on QASMBench circuits (Table 3,
# ratios of summed runtimes), not amplitude-updates/s, so no ratio is
# computed against them.
PAPER_CONTEXT = {
    "hardware": "16 Intel i7 cores at 2.50 GHz, 128 GB RAM (CPU only)",
    "speedup_full": {"vs_qulacs": 1.46, "vs_qiskit": 1.71},
    "speedup_incremental": {"vs_qulacs": 5.77, "vs_qiskit": 9.76},
    "source": "Table 3 (20 QASMBench circuits, block size 256, 16 threads)",
}


def make_workload(seed, rounds):
    from paper_2210_01076_gb300 import workloads as W
    levels = W.random_circuit(N_QUBITS, N_GATES, seed=seed, p_multi=P_MULTI)
    model = W.CircuitModel.from_levels(N_QUBITS, [list(lv) for lv in levels])
    stream_model = W.CircuitModel.from_levels(N_QUBITS, [list(lv) for lv in levels])
    edits = list(W.edit_stream(stream_model, rounds, seed=seed + 1, p_multi=P_MULTI))
    return levels, model, stream_model, edits


# Arithmetic peaks from unit counts and the maximum SM clock: SMs (read from
# the device) x 128 binary32 lanes x the maximum SM clock issue one binary32
# instruction each per cycle; binary64 FMA throughput is the measured 593 G/s
# of this GB300 (about 1.9 per cycle per SM of 152).  Float-float arithmetic
# is counted in binary32 instructions.
SM_COUNT, SM_MAX_GHZ = 152, 2.07
FP32_PEAK_TOPS = SM_COUNT * 128 * SM_MAX_GHZ / 1e3
FP64_PEAK_TOPS = 0.593


def set_device_peaks(dev_index=0):
    """The SM count of the device in use and the maximum SM clock
    (MEASURED_PEAKS.json's, else the GB300's 2070 MHz) set the binary32
    issue roof; the binary64 roof scales with the SM count."""
    global SM_COUNT, SM_MAX_GHZ, FP32_PEAK_TOPS, FP64_PEAK_TOPS
    try:
        import torch
        SM_COUNT = int(torch.cuda.get_device_properties(dev_index).multi_processor_count)
    except Exception:
        pass
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            SM_MAX_GHZ = float(json.load(f)["sm_max_mhz"]) / 1e3
    except Exception:
        pass
    FP32_PEAK_TOPS = SM_COUNT * 128 * SM_MAX_GHZ / 1e3
    FP64_PEAK_TOPS = 0.593 * SM_COUNT / 152


def roofline_pair(hbm_achieved, hbm_peak, peak_kind, alu_ops, kern_ms, dtype, traffic, launches, bytes_per_unit):
    """The fused-pass kernel against both roofs; the primary entry is the
    binding one (the larger fraction)."""
    hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
           "frac": (hbm_achieved / hbm_peak) if hbm_achieved else None, "peak_source": peak_kind,
           "traffic": traffic, "bytes_per_unit": bytes_per_unit}
    alu_peak = FP64_PEAK_TOPS if dtype == "c128" else FP32_PEAK_TOPS
    alu_ach = (alu_ops / (kern_ms * 1e-3) / 1e12) if kern_ms and kern_ms > 0 else None
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak,
           "unit": "T binary64 ops/s" if dtype == "c128" else "T binary32 ops/s",
           "frac": (alu_ach / alu_peak) if alu_ach else None,
           "peak_source": (f"unit counts x max SM clock ({SM_COUNT} SMs x 128 lanes x {SM_MAX_GHZ:.2f} GHz)"
                           if dtype != "c128" else f"measured FP64 FMA rate ({SM_COUNT} SMs)"),
           "sm_count": SM_COUNT,
           "ops_per_unit": "float-float: 86 binary32 ops per amplitude for a complex 2x2, 38 for a real 2x2, "
                           "diagonal or complex multiply" if dtype == "c128df" else "8 per complex 2x2 row, 4 real/mul"}
    primary = alu if (alu["frac"] or 0) > (hbm["frac"] or 0) else hbm
    other = hbm if primary is alu else alu
    out = dict(primary)
    out.update({"traffic": traffic, "kernel": "k_pass_reg / k_pass_tma (fused tile pass)", "kernel_ms_total": kern_ms,
                "kernel_launches": launches, "other_roof": other})
    return out


def config_dict(world):
    return {"workload": WORKLOAD, "n_qubits": N_QUBITS, "gates": N_GATES, "log2_partition": LOG2_PART,
            "ckpt_interval_levels": CKPT, "edits_per_round": "1-5", "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2: state 256 MiB, checkpoints ~5 GiB; no flush"}


def pctl(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if xs else None


# ------------------------------------------------------------------ ours --

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import build as qbuild

    rank, world, local_rank = rank_info()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    set_device_peaks(local_rank)
    qbuild.build()
    B.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)

    seed = rank_seed(rank)
    rounds = args.warmup + args.steps
    levels, _, final_model, edits = make_workload(seed, 2 * rounds + 2)

    c = B.Circuit(N_QUBITS, "c128df", LOG2_PART)
    c.set_stream(stream.cuda_stream)
    c.set_option("ckpt_interval", CKPT)
    for kv in args.option:
        k, v = kv.split("=")
        c.set_option(k, int(v))
    ids = c.load_levels(levels)
    h2id, k = {}, 0
    for lv in ids:
        for gid in lv:
            h2id[k] = gid
            k += 1
    full0 = c.update_state()  # initial full simulation (fills every checkpoint)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up rounds
    ri = 0
    for _ in range(args.warmup):
        B.apply_edit_ops(c, edits[ri], h2id)
        c.update_state()
        ri += 1

    # ---- timed: K incremental rounds, device time via CUDA events on the library's stream
    c.set_option("kernel_timing", 1)
    stats = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            B.apply_edit_ops(c, edits[ri], h2id)
            stats.append(c.update_state())
            ri += 1
        ev1.record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    elapsed_ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    amp = sum(s["amp_updates"] for s in stats)
    hbm = sum(s["hbm_bytes"] for s in stats)
    launches = sum(s["launches"] for s in stats)
    kern_ms = sum(s["pass_kernel_ms"] for s in stats)
    kern_bytes = sum(s["pass_kernel_bytes"] for s in stats)
    alu_ops = sum(s["pass_kernel_alu_ops"] for s in stats)
    kern_launches = sum(s["pass_kernel_launches"] for s in stats)
    amp_all, t_max_s = aggregate_over_ranks(amp, elapsed_ms * 1e-3, dev)
    t_max = t_max_s * 1e3
    value = amp_all / t_max_s

    # ---- full re-simulation latency on the current circuit (same plan),
    # timed like the rounds (with the per-launch events of kernel_timing)
    fulls, full_passes = [], 0
    for _ in range(3):
        fs = c.update_state(force_full=True)
        fulls.append(fs["gpu_ms"])
        full_passes = fs["passes_total"]
    c.set_option("kernel_timing", 0)
    inc_lat = [s["gpu_ms"] for s in stats]
    # per-round incremental efficiency: the round's time over what a full
    # re-simulation of that round's circuit costs for the work left dirty
    # (1 = the update costs exactly its dirty fraction of a full run).  The
    # circuit changes a little every round, so a round's full cost is the
    # measured full time scaled by its pass count.  Rounds with nothing dirty
    # (no work) have no efficiency and are counted apart.
    full_p50 = pctl(fulls, 50)
    eff, noop = [], 0
    for s in stats:
        dirty = (1.0 - s["clean_fraction"]) * full_p50 * s["passes_total"] / max(full_passes, 1)
        if s["passes_run"] == 0 or dirty <= 0.0:
            noop += 1
            continue
        eff.append(s["gpu_ms"] / dirty)

    # ---- end to end through the public API with host buffers: edits in,
    # update, the whole state read back to pinned host memory, every step.
    # The read of step k (qt_read_amplitudes_async: device snapshot, then a
    # copy on a second stream) overlaps the edits and update of step k+1; two
    # pinned buffers alternate, and the last copy is waited for inside the
    # timed region.
    host_bufs = [torch.empty((1 << N_QUBITS,), dtype=torch.complex128).pin_memory() for _ in range(2)]
    host_nps = [b.numpy() for b in host_bufs]
    e2e_amp, e2e_h2d = 0, 0
    e2e_rounds = 0 if args.no_e2e else min(args.steps, max(1, len(edits) - ri))
    barrier()
    te0 = time.perf_counter()
    for k in range(e2e_rounds):
        B.apply_edit_ops(c, edits[ri], h2id)
        s = c.update_state()
        c.read_wait()  # the previous step's copy has landed before its buffer is reused
        c.read_amplitudes_async(host_nps[k % 2])
        e2e_amp += s["amp_updates"]
        e2e_h2d += s["h2d_bytes"]
        ri += 1
    c.read_wait()
    barrier()
    te = time.perf_counter() - te0
    e2e_all, te_max = aggregate_over_ranks(e2e_amp, te, dev)
    e2e_val = e2e_all / te_max if e2e_rounds else None

    # ---- accuracy of the final state against the oracle (rank 0; the
    # oracle's state after the same rounds), and the norm
    accuracy = None
    norm = c.norm()
    if rank == 0 and not args.no_oracle_check:
        import oracle
        from paper_2210_01076_gb300 import workloads as W
        model = W.CircuitModel.from_levels(N_QUBITS, [list(lv) for lv in levels])
        rng_model = list(W.edit_stream(model, ri, seed=seed + 1, p_multi=P_MULTI))
        assert len(rng_model) == ri
        want = oracle.simulate(N_QUBITS, model.gates(), nthreads=oracle.max_threads())
        got = c.read_amplitudes()
        accuracy = {"max_abs_err_vs_fp64_oracle": float(np.max(np.abs(got - want))),
                    "fidelity": float(abs(np.vdot(want, got)) ** 2), "norm": norm, "tolerance": 1e-12}

    peak, peak_kind = measured_peak()
    achieved = (kern_bytes / (kern_ms * 1e-3)) / 1e9 if kern_ms > 0 else None
    khash = kernel_source_hash()
    traffic = profiled_traffic(khash)
    traffic_per_launch = None
    if traffic and kern_launches:
        # ncu DRAM bytes per unit (amplitude-pass), scaled to this run's average launch
        traffic_per_launch = traffic["dram_bytes_per_amp_pass"] * (kern_bytes / 32.0) / kern_launches

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(levels, budget_s=args.cpu_seconds)
    c.close()
    configs = None
    if rank == 0 and not args.no_configs:
        configs = run_configs(args, levels)

    if rank == 0:
        line = {
            "metric": "amplitude-updates/s",
            "value": value,
            "unit": "amp-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "c128 (float-float arithmetic)",
            "data": "synthetic (seeded random circuits and edit streams)",
            "config": config_dict(world),
            "hbm_gbs": hbm / (t_max * 1e-3) / 1e9,
            "incremental_latency_ms": {"p50": pctl(inc_lat, 50), "p99": pctl(inc_lat, 99)},
            "full_resim_latency_ms": {"p50": pctl(fulls, 50), "p99": pctl(fulls, 99)},
            "initial_full_sim_ms": full0["gpu_ms"],
            "clean_fraction_mean": float(np.mean([s["clean_fraction"] for s in stats])),
            "speedup_vs_full_p50": (pctl(fulls, 50) / pctl(inc_lat, 50)) if inc_lat else None,
            "incremental_efficiency": {
                "p50": pctl(eff, 50), "p99": pctl(eff, 99), "max": max(eff) if eff else None,
                "rounds_without_work": noop,
                "definition": "per round: incremental update time / ((1 - clean fraction) x full re-simulation "
                              "time of that round's circuit, the measured full time scaled by its pass count)",
                "rounds": [{"ms": s["gpu_ms"], "clean": s["clean_fraction"], "passes_run": s["passes_run"],
                            "passes_total": s["passes_total"], "launches": s["launches"]} for s in stats]},
            "accuracy": accuracy,
            "gpu_launches": launches,
            "roofline": roofline_pair(achieved, peak, peak_kind, alu_ops, kern_ms, "c128df", traffic_per_launch,
                                      kern_launches, "32 B per amplitude per pass (read + write of 16 B)"),
            "e2e": {"value": e2e_val, "unit": "amp-updates/s", "h2d_bytes_per_step": e2e_h2d / max(e2e_rounds, 1),
                    "d2h_bytes_per_step": (1 << N_QUBITS) * 16, "steps": e2e_rounds,
                    "note": "edits in, qt_update_state, whole state read to pinned host memory each step (qt_read_amplitudes_async: the copy of step k overlaps step k+1; the last is waited for in the timed region)"},
            "clocks": clocks,
            "wall_s_timed": t_wall,
            "paper_context": PAPER_CONTEXT,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if configs is not None:
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def host_record():
    """The host cores the oracle runs on: model name (from /proc/cpuinfo or
    lscpu) and the number of online CPUs."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "machine": os.uname().machine}


def cpu_baseline(levels, budget_s=15.0, gates_cap=None, n=None, keep=None):
    """The FP64 oracle on the host cores: a prefix of the workload's circuit at
    full size, gate by gate, until the time budget is spent.  With a dict
    `keep`, the oracle's state and the gates it applied are left in it."""
    import oracle
    from paper_2210_01076_gb300 import workloads as W
    n = N_QUBITS if n is None else n
    gates = W.flatten(levels)
    nth = oracle.max_threads()
    psi = np.zeros(1 << n, np.complex128)
    psi[0] = 1.0
    done = 0
    t0 = time.perf_counter()
    for g in gates:
        oracle.apply_gate(psi, g, nthreads=nth)
        done += 1
        if time.perf_counter() - t0 > budget_s or (gates_cap and done >= gates_cap):
            break
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.update(psi=psi, gates=gates[:done])
    return {"value": done * (1 << n) / dt, "unit": "amp-updates/s", "cores": nth, "kind": "oracle",
            "sample": f"first {done} gates of the n={n} circuit, full state, FP64 textbook loops ({dt:.1f} s)",
            "host": host_record()}


def oracle_prefix_accuracy(B, W, n, p, dtype, keep, tol):
    """The library against the FP64 oracle on the prefix of the circuit that
    the oracle simulated for the CPU baseline: the same gates in a fresh
    circuit, one full update, the max-abs amplitude error over the whole
    state (read back in chunks)."""
    psi, gates = keep["psi"], keep["gates"]
    c = B.Circuit(n, dtype, p)
    try:
        c.set_option("ckpt_interval", 1 << 20)  # one segment: state + output only
        c.load_levels(W.asap_levels(n, gates))
        c.update_state()
        err, chunk = 0.0, 1 << 24
        for first in range(0, 1 << n, chunk):
            cnt = min(chunk, (1 << n) - first)
            a = c.read_amplitudes(first, cnt).astype(np.complex128)
            err = max(err, float(np.max(np.abs(a - psi[first:first + cnt]))))
    finally:
        c.close()
    return {"gates": len(gates), "max_abs_err_vs_fp64_oracle": err, "tolerance": tol,
            "note": "the oracle's prefix of the circuit (the CPU-baseline sample), whole state"}


# ---------------------------------------------------------- other configs --
# Compact fixed-setting runs of the other workloads, reported under "configs"
# in the default line (each in seconds; no autotuning): the plain full
# simulation (n = 12), the deep QFT-like circuit (n = 30, both dtypes), the
# 256-circuit batch, a short served stream, and IEEE binary64 on the
# incremental workload's circuit.  A block that fails records its error and
# leaves the headline line intact.

def _guard(fn, *a, **k):
    try:
        return fn(*a, **k)
    except Exception as ex:  # the headline must survive a failing side block
        return {"error": f"{type(ex).__name__}: {ex}"}


def config1_block(B, W):
    """n = 12, 200 gates uniform over the 14 kinds, partitions of 2^8, one
    segment: full-simulation latency (the state is 64 KiB: L2-resident, bound
    by launches, not HBM), float-float and IEEE binary64, whole state against
    the FP64 oracle."""
    import oracle
    n, ng, p = 12, 200, 8
    levels = W.random_circuit(n, ng, seed=SEED, p_multi=None)
    want = oracle.simulate(n, W.flatten(levels))
    out = {"workload": f"plain full simulation n={n}, {ng} gates (14 kinds uniform), partitions 2^{p}"}
    for dt in ("c128df", "c128"):
        c = B.Circuit(n, dt, p)
        c.set_option("ckpt_interval", 1 << 20)
        c.load_levels(levels)
        c.update_state()
        sts = [c.update_state(force_full=True) for _ in range(30)]
        ms = [x["gpu_ms"] for x in sts]
        err = float(np.max(np.abs(c.read_amplitudes() - want)))
        c.close()
        out[dt] = {"full_sim_ms": {"p50": pctl(ms, 50), "p99": pctl(ms, 99)},
                   "host_ms_p50": pctl([x["host_ms"] for x in sts], 50),
                   "amp_updates_per_s": ng * (1 << n) / (pctl(ms, 50) * 1e-3),
                   "passes": sts[-1]["passes_total"], "launches": sts[-1]["launches"],
                   "accuracy": {"max_abs_err_vs_fp64_oracle": err, "tolerance": 1e-12, "whole_state": True}}
    return out


def _tail_edits(B, W, c, ids, levels, count, seed):
    rng = np.random.default_rng(seed)
    inc = []
    while len(inc) < count:
        e = W.tail_edit(rng, levels)
        if e is None:
            continue
        lvl, k, ng = e
        ids[lvl][k] = c.replace_gate(lvl, ids[lvl][k], ng)
        levels[lvl][k] = ng
        inc.append(c.update_state())
    return inc


def config3_block(B, W, peak, peak_kind):
    """n = 30, 2000 gates of QFT-like ladders and U3/CZ layers, partitions of
    2^18, fusion width 5 (the autotuner's choice), checkpoints sized from a
    device budget; a full simulation and 5 single-gate edits in the last 10 %
    of the levels, complex64 and float-float complex128.  Accuracy: the
    complex64 result against the float-float one over all 2^30 amplitudes
    (on the device); the float-float path's own error against the FP64
    oracle is measured on the incremental workload's whole state."""
    n, p, ng = 30, 18, 2000
    base = W.qft_like_circuit(n, ng, seed=7)
    out = {"workload": f"QFT-like n={n}, {ng} gates, partitions 2^{p}, fusion width 5, 5 tail edits"}
    # unfused HBM view first (its circuits are freed before the fused ones)
    for dt in ("c64", "c128df"):
        out.setdefault(dt, {})["unfused"] = deep30_unfused(B, W, n, p, dt, base, peak, 64)
    kept = {}
    try:
        for dt, budget_gb in (("c64", 64.0), ("c128df", 120.0)):
            levels = [list(x) for x in base]
            c = B.Circuit(n, dt, p)
            c.set_option("tile_high", 5)
            c.set_option("ckpt_budget", int(budget_gb * 1e9))
            ids = c.load_levels(levels)
            c.update_state()
            c.set_option("kernel_timing", 1)
            full = c.update_state(force_full=True)
            c.set_option("kernel_timing", 0)
            inc = _tail_edits(B, W, c, ids, levels, 5, seed=11)
            kept[dt] = c
            bpa = 8 if dt == "c64" else 16
            kb, km = full["pass_kernel_bytes"], full["pass_kernel_ms"]
            achieved = kb / (km * 1e-3) / 1e9 if km > 0 else None
            traffic = None
            t = profiled_traffic(kernel_source_hash(), "k_pass_c64_traffic.json" if dt == "c64" else
                                 "k_pass_df_traffic.json")
            if t and full["pass_kernel_launches"]:
                # ncu DRAM bytes per amplitude-pass (a smaller capture of the
                # same kernel), scaled to this run's average launch
                traffic = t["dram_bytes_per_amp_pass"] * (kb / (2 * bpa)) / full["pass_kernel_launches"]
            out[dt].update({
                "full_sim_ms": full["gpu_ms"], "amp_updates_per_s": full["amp_updates"] / (full["gpu_ms"] * 1e-3),
                "hbm_gbs": full["hbm_bytes"] / (full["gpu_ms"] * 1e-3) / 1e9,
                "segments": full["segments_total"], "passes": full["passes_total"], "ckpt_budget_gb": budget_gb,
                "incremental_ms": {"p50": pctl([x["gpu_ms"] for x in inc], 50),
                                   "p99": pctl([x["gpu_ms"] for x in inc], 99)},
                "clean_fraction_mean": float(np.mean([x["clean_fraction"] for x in inc])),
                "roofline": roofline_pair(achieved, peak, peak_kind, full["pass_kernel_alu_ops"], km, dt, traffic,
                                          full["pass_kernel_launches"], f"{2 * bpa} B per amplitude per pass")})
            if dt == "c64":
                out["c64_tensor_blocks"] = _guard(config3_tensor_blocks, B, W, base, c, full["gpu_ms"])
        c64, df = kept["c64"], kept["c128df"]
        out["c64"]["accuracy"] = {
            "max_abs_vs_c128df_whole_state": c64.max_abs_diff(df), "fidelity_vs_c128df": c64.fidelity(df),
            "norm": c64.norm(), "tolerance": {"max_abs": 1e-5, "fidelity": 1 - 1e-6},
            "note": "both after the same full simulation and 5 tail edits; the float-float reference is within "
                    "1e-12 of the FP64 oracle"}
        out["c128df"]["accuracy"] = {"norm": df.norm(), "tolerance": 1e-12,
                                     "note": "float-float error against the FP64 oracle: the headline's whole-state "
                                             "check and --workload deep30 --deep-oracle-full"}
    finally:
        for c in kept.values():
            c.close()
    return out


def config3_tensor_blocks(B, W, base, c64_ref, ref_ms, threshold=60):
    """The same complex64 circuit with runs of gates on five tile qubits
    folded into tensor-core blocks (tcgen05, 3xTF32) where the register
    kernel's estimate for the run exceeds `threshold` tenths of a dense op:
    full-simulation time against the register-only run, blocks launched,
    and the largest amplitude difference from the register-only state."""
    n, p = 30, 18
    levels = [list(x) for x in base]
    c = B.Circuit(n, "c64", p)
    try:
        c.set_option("tile_high", 5)
        c.set_option("ckpt_budget", int(64e9))
        c.set_option("tc_blocks", 1)
        c.set_option("tc_threshold", threshold)
        ids = c.load_levels(levels)
        c.update_state()
        c.set_option("kernel_timing", 1)  # as the register-only run was timed
        full = c.update_state(force_full=True)
        c.set_option("kernel_timing", 0)
        _tail_edits(B, W, c, ids, levels, 5, seed=11)
        return {"tc_threshold_tenths": threshold, "full_sim_ms": full["gpu_ms"],
                "register_only_full_sim_ms": ref_ms, "tensor_blocks_per_full_sim": full["tensor_blocks"],
                "max_abs_vs_register_path": c.max_abs_diff(c64_ref)}
    finally:
        c.close()


def config4_block(B, W):
    """256 complex64 circuits of 10-20 qubits and depths 50-400, one
    persistent launch, fusion width 5, then 3 rounds of one RZ/RY angle edit
    per circuit replayed from the captured CUDA graph; the smallest and the
    largest circuit against the oracle after the last round."""
    import oracle
    rng = np.random.default_rng(404)
    circs, levels, ids = [], [], []
    for n, lvls in W.batch_circuits(256, rng):
        c = B.Circuit(n, "c64", min(n, 16))
        c.set_option("tile_high", 5)
        ids.append(c.load_levels(lvls))
        levels.append([list(x) for x in lvls])
        circs.append(c)
    batch = B.Batch(circs)
    try:
        first = batch.run()
        capture = batch.run()
        rounds = []
        for _ in range(3):
            for k, c in enumerate(circs):
                e = W.rotation_edit(rng, levels[k])
                if e is None:
                    continue
                l, j, ng = e
                ids[k][l][j] = c.replace_gate(l, ids[k][l][j], ng)
                levels[k][l][j] = ng
            rounds.append(batch.run())
        acc = []
        for k in (int(np.argmin([c.n for c in circs])), int(np.argmax([c.n for c in circs]))):
            got = batch.read_amplitudes(k).astype(np.complex128)
            want = oracle.simulate(circs[k].n, W.flatten(levels[k]), nthreads=oracle.max_threads())
            acc.append({"qubits": circs[k].n, "gates": len(W.flatten(levels[k])),
                        "max_abs_err_vs_fp64_oracle": float(np.max(np.abs(got - want))),
                        "fidelity": float(abs(np.vdot(want, got)) ** 2 / np.vdot(got, got).real)})
        ms = [r["gpu_ms"] for r in rounds]
        return {"workload": "batch of 256 complex64 circuits, 10-20 qubits, depth 50-400, fusion width 5",
                "round_ms": {"p50": pctl(ms, 50), "p99": pctl(ms, 99)}, "first_run_ms": first["gpu_ms"],
                "capture_run_ms": capture["gpu_ms"], "graph_replays": int(sum(r["graph_replayed"] for r in rounds)),
                "amp_updates_per_s": rounds[-1]["amp_updates"] / (np.median(ms) * 1e-3),
                "tiles_per_launch": rounds[-1]["tiles"], "passes": rounds[-1]["passes"],
                "accuracy": {"circuits": acc, "tolerance": {"max_abs": 1e-5, "fidelity": 1 - 1e-6},
                             "whole_state": True}}
    finally:
        batch.close()
        for c in circs:
            c.close()


def ieee_c128_block(B, W, levels):
    """IEEE binary64 (QT_C128) on the incremental workload's circuit (n = 24,
    1000 gates, partitions 2^16, checkpoints every 8 levels): full
    re-simulation time against the float-float path of the same circuit,
    with the fused pass against the binary64 FMA roof."""
    out = {"workload": "incremental workload's circuit, full re-simulation"}
    for dt in ("c128", "c128df"):
        c = B.Circuit(N_QUBITS, dt, LOG2_PART)
        c.set_option("ckpt_interval", CKPT)
        c.load_levels(levels)
        c.update_state()
        c.set_option("kernel_timing", 1)
        sts = [c.update_state(force_full=True) for _ in range(3)]
        c.close()
        st = min(sts, key=lambda x: x["gpu_ms"])
        km = st["pass_kernel_ms"]
        alu = st["pass_kernel_alu_ops"] / (km * 1e-3) / 1e12 if km > 0 else None
        peak = FP64_PEAK_TOPS if dt == "c128" else FP32_PEAK_TOPS
        out[dt] = {"full_sim_ms": st["gpu_ms"], "amp_updates_per_s": st["amp_updates"] / (st["gpu_ms"] * 1e-3),
                   "pass_kernel_ms": km,
                   "hbm_gbs_kernel": st["pass_kernel_bytes"] / (km * 1e-3) / 1e9 if km > 0 else None,
                   "alu": {"achieved": alu, "peak": peak, "frac": alu / peak if alu else None,
                           "unit": "T binary64 FMA-class ops/s" if dt == "c128" else "T binary32 ops/s"}}
    out["float_float_speedup"] = out["c128"]["full_sim_ms"] / out["c128df"]["full_sim_ms"]
    return out


def precision_block(B, W):
    """The complex64 precision policy on two circuits: a 24-qubit QFT-like
    circuit of 2000 gates (amplitudes ~2^-12: the complex64 error stays far
    inside the contract) and a 5-qubit circuit of 50 000 random gates
    (amplitudes ~0.2: binary32 rounding carries the error past half the
    max-abs tolerance).  For each: the dtype the policy ends in, the error it
    measured against the float-float shadow, and the final error against
    the FP64 oracle over the whole state."""
    import oracle
    from paper_2210_01076_gb300.precision import AdaptiveCircuit
    out = {}
    for name, n, levels in (("qft_like_n24_2000", 24, W.qft_like_circuit(24, 2000, seed=7)),
                            ("random_n5_50000", 5, W.random_circuit(5, 50000, seed=5, p_multi=0.4))):
        ac = AdaptiveCircuit(n, min(n, 16), ckpt_interval=1 << 20)
        try:
            ac.load_levels(levels)
            t0 = time.perf_counter()
            ac.update_state()
            dt = time.perf_counter() - t0
            got = ac.read_amplitudes().astype(np.complex128)
            want = oracle.simulate(n, W.flatten(levels), nthreads=oracle.max_threads())
            rec = ac.error.get("switched_from_c64", ac.error)
            out[name] = {"final_dtype": ac.dtype, "switched": ac.switched_at_update is not None,
                         "measured_c64_max_abs": rec.get("max_abs"), "measured_c64_infidelity": rec.get("infidelity"),
                         "final_max_abs_err_vs_fp64_oracle": float(np.max(np.abs(got - want))),
                         "update_with_check_s": dt}
        finally:
            ac.close()
    out["policy"] = "switch to float-float complex128 when the measured complex64 error exceeds half of 1e-5 max-abs or 1e-6 infidelity"
    return out


def sharing_block(B, W, levels):
    """What a copy-on-write checkpoint store (Section III-F) could share: the
    mean fraction of partitions that a segment leaves unchanged
    (qt_segment_touched, planned on the host with dry runs), at the
    benchmarks' checkpoint spacings and at one level per checkpoint (the
    paper's per-net state vectors)."""
    def untouched(n, dtype, p, lv, G):
        c = B.Circuit(n, dtype, p)
        c.set_option("dry_run", 1)
        c.set_option("ckpt_interval", G)
        c.load_levels(lv)
        c.update_state()
        S = c.num_segments()
        frac = float(np.mean([1.0 - c.segment_touched(s).mean() for s in range(S)]))
        c.close()
        return {"levels_per_checkpoint": G, "segments": S, "unchanged_partition_fraction": frac}
    qft = W.qft_like_circuit(30, 2000, seed=7)
    return {"incremental_n24": [untouched(N_QUBITS, "c128df", LOG2_PART, levels, G) for G in (1, CKPT)],
            "qft_like_n30": [untouched(30, "c64", 18, qft, G) for G in (1, 8)],
            "note": "partitions a segment leaves unchanged could be shared with the previous checkpoint"}


def run_configs(args, levels):
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import workloads as W
    peak, peak_kind = measured_peak()
    t0 = time.perf_counter()
    out = {}
    out["plain_full_n12"] = _guard(config1_block, B, W)
    out["ieee_binary64_n24"] = _guard(ieee_c128_block, B, W, levels)
    out["deep_qft_n30"] = _guard(config3_block, B, W, peak, peak_kind)
    out["batch256"] = _guard(config4_block, B, W)
    out["precision_policy"] = _guard(precision_block, B, W)
    out["checkpoint_sharing"] = _guard(sharing_block, B, W, levels)
    if args.configs_serve:
        sargs = argparse.Namespace(**vars(args))
        sargs.serve_seconds, sargs.serve_burst, sargs.serve_check = 1.0, 100, 0
        out["serve64"] = _guard(run_serve, sargs, emit=False)
    out["wall_s"] = time.perf_counter() - t0
    return out


# ------------------------------------------------------------- reference --

def run_deep30(args):
    """The large deep-circuit configuration: n = 30, 2000 gates of QFT-style
    H + controlled-phase ladders interleaved with U3/CZ layers, complex64 or
    complex128 (float-float); a full simulation, then single-gate edits in the
    last 10 % of the levels, each followed by an incremental update.  Prints
    its own JSON line (not the default benchmark)."""
    import torch
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import build as qbuild
    from paper_2210_01076_gb300 import workloads as W
    qbuild.build()
    B.load()
    set_device_peaks(0)
    from paper_2210_01076_gb300 import tuning
    n, ngates = args.deep_n, 2000
    p = min(18, n)
    dtype = args.dtype
    levels = W.qft_like_circuit(n, ngates, seed=7)
    tuned = None
    if args.deep_tune:
        # the fusion width (qubits a tile holds above its low run), timed 1..5
        # on full simulations without checkpoints; the best one is used below
        t = tuning.tune_circuit(n, dtype, levels, p, tile_high=range(1, 6), ckpt_interval=(1 << 20,),
                                merge=(1,), repeats=1)
        if t["best"]:
            tuned = {"tile_high": t["best"]["options"]["tile_high"],
                     "full_ms": {str(r["options"]["tile_high"]): r.get("full_ms") for r in t["table"]}}
    stream = torch.cuda.Stream()
    c = B.Circuit(n, dtype, p)
    c.set_stream(stream.cuda_stream)
    if tuned:
        c.set_option("tile_high", tuned["tile_high"])
    ckpt = args.deep_ckpt
    c.set_option("ckpt_interval", ckpt)
    if args.deep_ckpt_budget_gb > 0:
        # as many checkpoints as the budget holds (the library sets the interval)
        c.set_option("ckpt_budget", int(args.deep_ckpt_budget_gb * 1e9))
    for kv in args.option:
        k, v = kv.split("=")
        c.set_option(k, int(v))
    ids = c.load_levels(levels)
    c.update_state()
    c.set_option("kernel_timing", 1)
    fulls = [c.update_state(force_full=True) for _ in range(2)]
    c.set_option("kernel_timing", 0)
    full = fulls[-1]
    rng = np.random.default_rng(11)
    L = len(levels)
    inc = []
    for _ in range(args.steps):
        # every edit changes the plan (a new RZ or CP angle)
        e = W.tail_edit(rng, levels)
        if e is None:
            continue
        lvl, k, ng = e
        ids[lvl][k] = c.replace_gate(lvl, ids[lvl][k], ng)
        levels[lvl][k] = ng
        inc.append(c.update_state())
    norm = c.norm()
    accuracy_full = deep30_whole_state_accuracy(B, W, c, n, p, dtype, levels, args.deep_oracle_full)
    peak, peak_kind = measured_peak()
    kb, km = full["pass_kernel_bytes"], full["pass_kernel_ms"]
    achieved = kb / (km * 1e-3) / 1e9 if km > 0 else None
    bpa = 8 if dtype == "c64" else 16
    traffic_per_launch = None
    if dtype == "c64" and full["pass_kernel_launches"]:
        # ncu DRAM bytes per amplitude-pass of the complex64 instantiation
        # (captured on a smaller state of the same circuit family), scaled to
        # this run's average launch
        t = profiled_traffic(kernel_source_hash(), "k_pass_c64_traffic.json")
        if t:
            traffic_per_launch = t["dram_bytes_per_amp_pass"] * (kb / (2 * bpa)) / full["pass_kernel_launches"]
    line = {
        "metric": "amplitude-updates/s", "workload": "deep30",
        "value": full["amp_updates"] / (full["gpu_ms"] * 1e-3), "unit": "amp-updates/s",
        "dtype": {"c64": "c64 (fp32)", "c128df": "c128 (float-float)", "c128": "c128 (fp64)"}[dtype],
        "config": {"workload": f"QFT-like n={n}, 2000 gates, partitions 2^{p}",
                   "ckpt_interval_levels": -(-L // full["segments_total"]) if args.deep_ckpt_budget_gb > 0 else ckpt,
                   "ckpt_budget_gb": args.deep_ckpt_budget_gb or None,
                   "levels": L, "segments": full["segments_total"], "passes": full["passes_total"],
                   "fusion_width_tuned": tuned},
        "full_sim_ms": full["gpu_ms"], "hbm_gbs": full["hbm_bytes"] / (full["gpu_ms"] * 1e-3) / 1e9,
        "incremental_latency_ms": {"p50": pctl([s["gpu_ms"] for s in inc], 50),
                                   "p99": pctl([s["gpu_ms"] for s in inc], 99)},
        "clean_fraction_mean": float(np.mean([s["clean_fraction"] for s in inc])) if inc else None,
        "norm": norm,
        "accuracy_whole_state": accuracy_full,
        "roofline": roofline_pair(achieved, peak, peak_kind, full["pass_kernel_alu_ops"], km, dtype, traffic_per_launch,
                                  full["pass_kernel_launches"], f"{2 * bpa} B per amplitude per pass"),
    }
    c.close()
    line["unfused"] = deep30_unfused(B, W, n, p, dtype, levels, peak, args.deep_unfused_gates)
    if args.deep_oracle_s > 0:
        keep = {}
        line["cpu_baseline"] = cpu_baseline(levels, budget_s=args.deep_oracle_s, n=n, keep=keep)
        line["accuracy"] = oracle_prefix_accuracy(B, W, n, p, dtype, keep, 1e-5 if dtype == "c64" else 1e-12)
        keep.clear()
    print(json.dumps(line), flush=True)


def deep30_whole_state_accuracy(B, W, c, n, p, dtype, levels, with_oracle):
    """The final state (after the full simulation and the tail edits) over
    all 2^n amplitudes: a complex64 result against a float-float run of the
    same gates (on the device); with `with_oracle`, the result -- and, for a
    complex64 run, the float-float reference too -- against the FP64
    oracle's full simulation of the same gates on the host cores (2000
    gates on 2^30 amplitudes: minutes on 16 cores, 16 GiB)."""
    out = {}
    ref = None
    try:
        if dtype == "c64":
            ref = B.Circuit(n, "c128df", p)
            ref.set_option("ckpt_interval", 1 << 20)
            ref.load_levels(levels)
            ref.update_state()
            out["vs_c128df"] = {"max_abs": c.max_abs_diff(ref), "fidelity": c.fidelity(ref),
                                "tolerance": {"max_abs": 1e-5, "fidelity": 1 - 1e-6}}
        if with_oracle:
            import oracle
            t0 = time.perf_counter()
            want = oracle.simulate(n, W.flatten(levels), nthreads=oracle.max_threads())
            t_or = time.perf_counter() - t0
            sides = [(dtype, c, 1e-5 if dtype == "c64" else 1e-12)]
            if ref is not None:
                sides.append(("c128df", ref, 1e-12))
            for name, circ, tol in sides:
                err, dot, na, chunk = 0.0, 0j, 0.0, 1 << 24
                for first in range(0, 1 << n, chunk):
                    cnt = min(chunk, (1 << n) - first)
                    a = circ.read_amplitudes(first, cnt).astype(np.complex128)
                    w = want[first:first + cnt]
                    err = max(err, float(np.max(np.abs(a - w))))
                    dot += np.vdot(w, a)
                    na += float(np.vdot(a, a).real)
                out[f"{name}_vs_fp64_oracle"] = {"max_abs": err, "fidelity": float(abs(dot) ** 2 / na),
                                                 "tolerance": tol}
            out["oracle"] = {"seconds": t_or, "threads": oracle.max_threads(), "gates": len(W.flatten(levels)),
                             "host": host_record()}
            del want
    finally:
        if ref is not None:
            ref.close()
    return out or None


def deep30_unfused(B, W, n, p, dtype, levels, peak, ngates):
    """The same kernel with fusion off: the first `ngates` gates of the
    circuit, one gate per pass, so that each pass is bound by HBM rather
    than by instruction issue.  Reports the passes' HBM bandwidth (bytes
    read and written per pass over the event-timed kernel time) against the
    measured peak, and the amplitude-update rate that fusion improves on."""
    if ngates <= 0:
        return None
    gates = W.flatten(levels)[:ngates]
    c = B.Circuit(n, dtype, p)
    c.set_option("fusion", 0)
    c.set_option("ckpt_interval", 1 << 20)
    c.load_levels(W.asap_levels(n, gates))
    c.update_state()
    c.set_option("kernel_timing", 1)
    st = min((c.update_state(force_full=True) for _ in range(2)), key=lambda s: s["pass_kernel_ms"])
    c.close()
    gbs = st["pass_kernel_bytes"] / (st["pass_kernel_ms"] * 1e-3) / 1e9
    return {"gates": len(gates), "passes": st["passes_total"], "kernel_ms": st["pass_kernel_ms"],
            "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / peak if peak else None,
            "amp_updates_per_s": st["amp_updates"] / (st["gpu_ms"] * 1e-3)}


def run_serve(args, emit=True):
    """Served request stream: 64 resident circuits of 16-28 qubits (complex64,
    300-1500 random gates), requests of 1-5 edits + an incremental update
    arriving as a Poisson stream, device memory admitted against a 150 GB
    budget including checkpoints.  Reports throughput and p50/p99 latency at
    the offered 2000 req/s and at 70 % of the measured capacity."""
    import threading
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import build as qbuild
    from paper_2210_01076_gb300 import workloads as W
    qbuild.build()
    B.load()
    rng = np.random.default_rng(55)
    ncirc = args.serve_circuits
    circs, mirrors, ids, ns = [], [], [], []
    for c in range(ncirc):
        n = int(rng.integers(16, 29))
        levels = W.random_circuit(n, int(rng.integers(300, 1501)), seed=5000 + c, p_multi=0.4)
        circ = B.Circuit(n, "c64", min(n, 16))
        circ.set_option("ckpt_interval", max(4, -(-len(levels) // 8)))  # at most ~9 checkpoints
        ids.append(circ.load_levels(levels))
        mirrors.append([list(lv) for lv in levels])
        circs.append(circ)
        ns.append(n)
    budget = int(args.serve_budget_gb * 1e9)
    srv = B.Server(workers=args.serve_workers, hbm_budget_bytes=budget)
    slots = [srv.add_circuit(c) for c in circs]
    t0 = time.perf_counter()
    for t in [srv.submit(s, []) for s in slots]:
        srv.wait(t)
    warm_s = time.perf_counter() - t0
    replaced = [set() for _ in range(ncirc)]

    def make_request():
        c = int(rng.integers(ncirc))
        ops = []
        for _ in range(int(rng.integers(1, 6))):
            if rng.random() < 0.5:
                lvl = int(rng.integers(len(mirrors[c]) + 1))
                g = W.random_gate(rng, ns[c], 0.4)
                ops += [("insert_level", lvl), ("insert", lvl, g)]
                mirrors[c].insert(lvl, [g])
                ids[c].insert(lvl, [None])
            else:
                cand = [(l, k) for l, lv in enumerate(ids[c]) for k, gid in enumerate(lv)
                        if gid is not None and gid not in replaced[c]]
                if not cand:
                    continue
                l, k = cand[int(rng.integers(len(cand)))]
                q = list(mirrors[c][l][k].qubits)
                same = [nm for nm in W.ALL_KINDS if sum(W.ARITY[nm][:2]) == len(q)]
                nm = same[int(rng.integers(len(same)))]
                ng = W.make_gate(nm, q, rng.uniform(0, 2 * np.pi, W.ARITY[nm][2]))
                ops.append(("replace", l, ids[c][l][k], ng))
                replaced[c].add(ids[c][l][k])
                mirrors[c][l][k] = ng
                ids[c][l][k] = None
        return c, ops

    def open_loop(rate, seconds):
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 1))
        arrivals = arrivals[arrivals < seconds]
        reqs = [make_request() for _ in arrivals]
        tickets, results = [], []
        done = threading.Event()

        def waiter():
            k = 0
            while k < len(arrivals):
                while len(tickets) <= k:
                    time.sleep(0.0005)
                results.append(srv.wait(tickets[k]))
                k += 1
            done.set()
        th = threading.Thread(target=waiter)
        th.start()
        start = time.perf_counter()
        for (c, ops), at in zip(reqs, arrivals):
            dt = start + at - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(slots[c], ops))
        th.join()
        wall = time.perf_counter() - start
        lat = [r["latency_ms"] for r in results]
        amp = sum(r["stats"]["amp_updates"] for r in results)
        # device time of every request's update (events on its circuit's
        # stream) summed over the window: above the wall time only if
        # requests' work overlapped on the device
        dev_ms = sum(max(r["stats"]["gpu_ms"], 0.0) for r in results)
        return {"offered_req_s": rate, "window_s": seconds, "requests": len(results), "wall_s": wall,
                "throughput_req_s": len(results) / wall, "amp_updates_per_s": amp / wall,
                "latency_ms": {"p50": pctl(lat, 50), "p99": pctl(lat, 99)},
                "device_ms_sum": dev_ms, "overlap_factor": dev_ms / (wall * 1e3),
                "queue_ms_p50": pctl([r["queue_ms"] for r in results], 50),
                "service_ms_p50": pctl([r["service_ms"] for r in results], 50),
                "errors": sum(1 for r in results if r["status"] != 0)}

    # capacity: a closed burst
    burst = [make_request() for _ in range(args.serve_burst)]
    tb = time.perf_counter()
    tickets = [srv.submit(slots[c], ops) for c, ops in burst]
    res = [srv.wait(t) for t in tickets]
    burst_wall = time.perf_counter() - tb
    cap = len(res) / burst_wall
    burst_dev_ms = sum(max(r["stats"]["gpu_ms"], 0.0) for r in res)
    at_2k = open_loop(2000.0, args.serve_seconds)
    at_70 = open_loop(0.7 * cap, args.serve_seconds)
    info = srv.info()
    srv.close()
    accuracy = serve_accuracy(B, circs, mirrors, ns, args.serve_check) if args.serve_check > 0 else None
    oracle_acc = serve_oracle_accuracy(B, circs, mirrors, ns, max_qubits=args.serve_oracle_max_n)
    line = {"metric": "served requests", "workload": "serve64", "dtype": "c64 (fp32)",
            "config": {"circuits": ncirc, "qubits": "16-28", "gates": "300-1500", "edits_per_request": "1-5",
                       "workers": args.serve_workers, "hbm_budget_gb": args.serve_budget_gb},
            "warmup_full_sims_s": warm_s, "capacity_req_s": cap,
            "capacity_burst": {"requests": len(res), "wall_s": burst_wall, "device_ms_sum": burst_dev_ms,
                               "overlap_factor": burst_dev_ms / (burst_wall * 1e3),
                               "device_ms_per_request_p50": pctl([r["stats"]["gpu_ms"] for r in res], 50),
                               "device_ms_per_request_mean": burst_dev_ms / max(len(res), 1)},
            "at_offered_2000": at_2k,
            "at_70pct_capacity": at_70, "evictions": info["evictions"],
            "resident_gb": info["resident_bytes"] / 1e9, "accuracy_vs_plain_c128": accuracy,
            "accuracy_vs_fp64_oracle": oracle_acc}
    for c in circs:
        c.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def serve_oracle_accuracy(B, circs, mirrors, ns, max_qubits=22):
    """The served complex64 states of every circuit of at most `max_qubits`
    qubits, after all requests, against the FP64 oracle over the whole state
    (the oracle takes seconds per circuit up to 22 qubits on the host cores)."""
    import oracle
    from paper_2210_01076_gb300 import workloads as W
    picks = sorted((c for c in range(len(circs)) if ns[c] <= max_qubits), key=lambda c: -ns[c])[:3]
    per, worst_err, worst_fid = [], 0.0, 1.0
    for c in picks:
        circs[c].update_state()  # re-simulates a circuit the server evicted (the same bits)
        got = circs[c].read_amplitudes().astype(np.complex128)
        want = oracle.simulate(ns[c], W.flatten(mirrors[c]), nthreads=oracle.max_threads())
        err = float(np.max(np.abs(got - want)))
        fid = float(abs(np.vdot(want, got)) ** 2 / (np.vdot(got, got).real * np.vdot(want, want).real))
        per.append({"qubits": ns[c], "gates": int(sum(len(lv) for lv in mirrors[c])), "max_abs_err": err,
                    "fidelity": fid})
        worst_err, worst_fid = max(worst_err, err), min(worst_fid, fid)
        circs[c].release_device()
    return {"circuits_checked": len(per), "max_abs_err": worst_err, "min_fidelity": worst_fid,
            "tolerance": {"max_abs": 1e-5, "fidelity": 1 - 1e-6}, "per_circuit": per, "whole_state": True}


def serve_accuracy(B, circs, mirrors, ns, count):
    """Accuracy of served results: for `count` of the circuits (the smallest,
    the largest, the rest drawn by seed) the served complex64 state after
    all requests against the plain unbatched complex128 (binary64) path run
    on the same edited circuit -- max-abs amplitude error and fidelity."""
    order = sorted(range(len(circs)), key=lambda c: ns[c])
    pick = [order[0], order[-1]]
    rest = [c for c in order[1:-1]]
    rng = np.random.default_rng(56)
    pick += [int(c) for c in rng.choice(rest, size=min(max(count - 2, 0), len(rest)), replace=False)]
    pick = pick[:count]
    for c, circ in enumerate(circs):
        if c not in pick:
            circ.release_device()
    worst_err, worst_fid, per = 0.0, 1.0, []
    for c in pick:
        circ = circs[c]
        circ.update_state()  # re-simulates a circuit the server evicted (the same bits)
        ref = B.Circuit(ns[c], "c128", min(ns[c], 16))
        ref.set_option("ckpt_interval", len(mirrors[c]) + 1)  # no checkpoints needed
        ref.load_levels(mirrors[c])
        ref.update_state()
        fid = circ.fidelity(ref)
        err, chunk = 0.0, 1 << 22
        for first in range(0, 1 << ns[c], chunk):
            cnt = min(chunk, (1 << ns[c]) - first)
            a = circ.read_amplitudes(first, cnt).astype(np.complex128)
            err = max(err, float(np.max(np.abs(a - ref.read_amplitudes(first, cnt)))))
        ref.close()
        circ.release_device()
        per.append({"qubits": ns[c], "gates": int(sum(len(lv) for lv in mirrors[c])), "max_abs_err": err,
                    "fidelity": fid})
        worst_err, worst_fid = max(worst_err, err), min(worst_fid, fid)
    return {"circuits_checked": len(per), "max_abs_err": worst_err, "min_fidelity": worst_fid,
            "tolerance": {"max_abs": 1e-5, "fidelity": 1 - 1e-6}, "per_circuit": per}


def run_batch(args):
    """Batched synthesis loop: 256 independent complex64 circuits, qubit
    counts uniform in [10, 20], depths (ASAP levels) uniform in [50, 400],
    simulated together in one persistent launch; then 10 rounds in which
    every circuit gets one parameter edit (an RZ or RY angle moved by
    N(0, 0.1)) and the batch re-runs (CUDA-graph replay)."""
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import build as qbuild
    from paper_2210_01076_gb300 import workloads as W
    qbuild.build()
    B.load()
    rng = np.random.default_rng(404)
    circs, levels, ids = [], [], []
    for n, lvls in W.batch_circuits(args.batch_circuits, rng):
        c = B.Circuit(n, "c64", min(n, 16))
        ids.append(c.load_levels(lvls))
        levels.append([list(x) for x in lvls])
        circs.append(c)
    tuned = None
    if args.batch_tune:
        # the fusion width of every circuit of the batch, timed 3..5
        from paper_2210_01076_gb300 import tuning
        t = tuning.tune_batch(circs, tile_high=(3, 4, 5))
        if t["best"]:
            tuned = {"tile_high": t["best"]["tile_high"],
                     "round_ms": {str(r["tile_high"]): r.get("round_ms") for r in t["table"]}}
    batch = B.Batch(circs)
    first = batch.run()
    capture = batch.run()
    rounds = []
    for _ in range(args.batch_rounds):
        for k, c in enumerate(circs):
            e = W.rotation_edit(rng, levels[k])
            if e is None:
                continue
            l, j, ng = e
            ids[k][l][j] = c.replace_gate(l, ids[k][l][j], ng)
            levels[k][l][j] = ng
        rounds.append(batch.run())
    # one circuit checked against the oracle after the last round
    import oracle
    k = int(np.argmin([c.n for c in circs]))
    err = float(np.max(np.abs(batch.read_amplitudes(k).astype(np.complex128)
                              - oracle.simulate(circs[k].n, W.flatten(levels[k])))))
    ms = [r["gpu_ms"] for r in rounds]
    amp = rounds[-1]["amp_updates"] if rounds else first["amp_updates"]
    line = {"metric": "amplitude-updates/s", "workload": "batch256", "dtype": "c64 (fp32)",
            "value": amp / (np.median(ms) * 1e-3), "unit": "amp-updates/s",
            "config": {"circuits": len(circs), "qubits": "10-20", "depth": "50-400",
                       "gates_total": int(sum(c.num_gates() for c in circs)), "passes": rounds[-1]["passes"],
                       "fusion_width_tuned": tuned,
                       "tiles_per_launch": rounds[-1]["tiles"]},
            "first_run_ms": first["gpu_ms"], "capture_run_ms": capture["gpu_ms"],
            "round_ms": {"p50": pctl(ms, 50), "p99": pctl(ms, 99)},
            "graph_replays": int(sum(r["graph_replayed"] for r in rounds)), "rounds": len(rounds),
            "max_abs_err_vs_oracle_smallest_circuit": err}
    print(json.dumps(line), flush=True)
    batch.close()


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    import oracle
    from paper_2210_01076_gb300 import workloads as W
    levels = W.random_circuit(N_QUBITS, N_GATES, seed=SEED, p_multi=P_MULTI)
    gates = W.flatten(levels)
    nth = oracle.max_threads()
    psi = np.zeros(1 << N_QUBITS, np.complex128)
    psi[0] = 1.0
    per_step = 8  # gates of the re-simulation sampled per step
    gi = 0
    for _ in range(args.warmup):
        for _ in range(per_step):
            oracle.apply_gate(psi, gates[gi % len(gates)], nthreads=nth)
            gi += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            oracle.apply_gate(psi, gates[gi % len(gates)], nthreads=nth)
            gi += 1
    dt = time.perf_counter() - t0
    value = args.steps * per_step * (1 << N_QUBITS) / dt
    line = {
        "impl": "reference", "metric": "amplitude-updates/s", "value": value, "unit": "amp-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded random circuits)",
        "config": config_dict(world),
        "cpu_baseline": {"value": value, "unit": "amp-updates/s", "cores": nth, "kind": "oracle",
                         "sample": f"{per_step} gates of the n=24 circuit per step (a CPU re-simulation "
                                   f"re-runs every gate after the edit)", "host": host_record()},
        "e2e": {"value": value, "unit": "amp-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    global N_QUBITS, CKPT
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations' compact runs")
    ap.add_argument("--configs-serve", type=int, default=1, help="include the short served stream in 'configs'")
    ap.add_argument("--serve-oracle-max-n", type=int, default=22,
                    help="serve: circuits up to this many qubits are checked against the FP64 oracle")
    ap.add_argument("--n-qubits", type=int, default=N_QUBITS, help="smaller cases for profiling only")
    ap.add_argument("--ckpt", type=int, default=CKPT, help="levels per checkpoint segment")
    ap.add_argument("--option", action="append", default=[], help="extra qt_set_option key=value")
    ap.add_argument("--workload", default="incremental24", choices=["incremental24", "deep30", "serve", "batch"])
    ap.add_argument("--batch-circuits", type=int, default=256)
    ap.add_argument("--batch-rounds", type=int, default=10)
    ap.add_argument("--batch-tune", type=int, default=1, help="batch: autotune the fusion width (tile_high 3..5)")
    ap.add_argument("--serve-circuits", type=int, default=64)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-burst", type=int, default=200)
    ap.add_argument("--serve-check", type=int, default=6,
                    help="served circuits checked against the plain complex128 path afterwards")
    ap.add_argument("--dtype", default="c128df", choices=["c128df", "c64", "c128"], help="deep30 only")
    ap.add_argument("--deep-ckpt", type=int, default=48, help="deep30: levels per checkpoint segment")
    ap.add_argument("--deep-ckpt-budget-gb", type=float, default=200.0,
                    help="deep30: device memory for the state and checkpoints (sets the interval); 0 = --deep-ckpt")
    ap.add_argument("--deep-tune", type=int, default=1, help="deep30: autotune the fusion width (tile_high 1..5)")
    ap.add_argument("--deep-oracle-s", type=float, default=15.0,
                    help="deep30: seconds of FP64 oracle on the host cores (a prefix of the circuit); 0 = skip")
    ap.add_argument("--deep-n", type=int, default=30, help="deep30: qubits (smaller cases for profiling only)")
    ap.add_argument("--deep-oracle-full", type=int, default=0,
                    help="deep30: 1 = also the FP64 oracle's whole 2000-gate simulation (minutes on the host cores)")
    ap.add_argument("--deep-unfused-gates", type=int, default=64,
                    help="deep30: gates timed one per pass (fusion off) for the HBM-bound view; 0 = skip")
    args = ap.parse_args()
    N_QUBITS, CKPT = args.n_qubits, args.ckpt
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "deep30":
        run_deep30(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
