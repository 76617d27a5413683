#!/usr/bin/env python3
"""Benchmark of the LS all-vs-all hot path: cell-updates/s (N^2 L per step) for forward +
backward + posterior + distance at D loci, on the dense FP32 workload N=5000, L=20000, D=16.

One step = one ls_run_all over the whole workload (both recursions over all loci, decoding at
the 16 loci, symmetrised N x N distances, PAC log-likelihood), inputs resident in HBM.  L2 is
flushed (a 256 MiB write, outside the timed events) before every timed step.  The propagation
kernels dominate; their roofline is the FP32 pipe (8 algorithmic FLOPs per cell-update: 4 in each
direction), against 2 x 128 x SMs x max SM clock.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]

Multi-GPU (torchrun): every rank runs its own replica of the workload (targets shard with no
exchange except the distance transpose, which this single-node benchmark does not exercise);
times are the max over ranks and `value` counts every rank's cell-updates.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LS cell-updates/s (N^2*L, fwd+bwd+distance)"
UNIT = "cell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ls_n5000_l20000")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample size, in seconds of CPU work")
    ap.add_argument("--cpu-threads", type=int, default=0, help="oracle threads (0: every host core)")
    ap.add_argument("--N", type=int, default=None, help="override N (small cases for profiling; not a bench line)")
    ap.add_argument("--L", type=int, default=None, help="override L (small cases for profiling; not a bench line)")
    ap.add_argument("--D", type=int, default=None, help="override the number of decode loci (profiling cases)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ls_prop_kernel_dram_n5000.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2212_11403_gb300", "csrc", f) for f in ("ls_prop.cuh", "ls_prop_inst.cu")]


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(N, L, D):
    """DRAM bytes per step of the propagation launches from the committed ncu summary: the captured
    bytes (same N and D, fewer loci) plus the extra packed-row reads of the longer run, or None when
    the summary was taken on other kernel sources or another workload shape."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256_16") != kernel_digest():
            return None
        if int(kv["N"]) != N or int(kv["D"]) != D:
            return None
        rows = float(kv["row_bytes_per_locus_per_pass"]) * 2 * (L - int(kv["L"]))
        return float(kv["dram_bytes_per_step"]) + rows
    except (OSError, KeyError, ValueError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def make_inputs(name, N=None, L=None):
    from paper_2212_11403_gb300 import synth
    w = synth.make_workload(name, N=N, L=L)
    if w["rho"] is None:
        from paper_2212_11403_gb300 import ls
        w["rho"] = ls.ls_calc_rho(w["gaps"], w["Ne"], 1.0)
    return w


def oracle_sample(w, seconds, seed=7, threads=0):
    """Time the FP64 oracle (as it stands) on a bounded sample of targets of the same workload."""
    import oracle
    N, L = w["N"], w["L"]
    rng = np.random.default_rng(seed)
    threads = threads if threads > 0 else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.run(w["h"], w["rho"], w["mu"], w["loci"], targets=rng.choice(N, size=1, replace=False), want=("llf",),
               nthreads=1)
    per_target = time.perf_counter() - t0
    n = int(max(threads, min(N, round(seconds * threads / max(per_target, 1e-6)))))
    n = min(N, max(threads, (n // threads) * threads))
    targets = np.sort(rng.choice(N, size=n, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    oracle.run(w["h"], w["rho"], w["mu"], w["loci"], targets=targets, want=("post", "llf"), nthreads=threads)
    dt = time.perf_counter() - t0
    return dict(value=n * N * L / dt, unit=UNIT, cores=threads, kind="oracle",
                sample="%d of %d targets (fwd+bwd over all %d loci, posteriors at %d loci), FP64 C, %d threads, "
                       "%.1f s" % (n, N, L, len(w["loci"]), threads, dt))


def run_reference(args, world, rank):
    """--impl reference: the FP64 oracle on the host cores, a bounded target sample per step."""
    if rank != 0:
        return
    w = make_inputs(args.workload, args.N, args.L)
    N, L = w["N"], w["L"]
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    samples = []
    for s in range(args.warmup + args.steps):
        r = oracle_sample(w, per_step, seed=100 + s, threads=args.cpu_threads)
        if s >= args.warmup:
            samples.append(r)
    vals = [r["value"] for r in samples]
    value = float(np.median(vals))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * float(N) * N * L / value, ms_per_step_basis="whole workload, extrapolated "
                "linearly in the number of targets from the timed sample", higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic founder mosaics (seeded)", impl="reference",
                config={"workload": args.workload, "N": N, "L": L, "D": int(len(w["loci"]))},
                cpu_baseline=dict(value=value, unit=UNIT, cores=samples[-1]["cores"], kind="oracle",
                                  sample=samples[-1]["sample"]),
                e2e={"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2212_11403_gb300 import ls

    w = make_inputs(args.workload, args.N, args.L)
    if args.D:
        from paper_2212_11403_gb300 import synth
        w["loci"] = synth.decode_loci(w["L"], args.D)
    N, L, loci = w["N"], w["L"], w["loci"]
    D = len(loci)
    cells = float(N) * N * L
    ctx = ls.ls_create(w["h"])
    ls.ls_set_params(ctx, w["rho"], w["mu"])
    d = torch.empty((D, N, N), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ls.ls_set_profiling(ctx, True)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        flush.zero_()
        ls.ls_run_all(ctx, loci, d, want_pac=False)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    step_ms, phase_ms, launches = [], [], 0
    pac = None
    for s in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, pac = ls.ls_run_all(ctx, loci, d, want_pac=(s == args.steps - 1))
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ms, nl = ls.ls_profile_read(ctx)
        phase_ms.append(ms)
        launches += int(sum(nl))
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()

    t_step = max_over_ranks(float(np.mean(step_ms)), world)
    value = world * cells / (t_step / 1e3)
    ph = np.mean(np.array(phase_ms), axis=0)
    t_prop = float(ph[0] + ph[1])  # forward + backward propagation launches
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    p_fp32 = 2 * 128 * nsm * sm_max * 1e6 / 1e12  # TFLOP/s at the maximum SM clock
    achieved = 8.0 * cells / (t_prop / 1e3) / 1e12
    traffic = dram_traffic(N, L, D)
    roof = dict(bound="alu", kernel="ls_prop_kernel (forward + backward launches)", achieved=achieved, peak=p_fp32,
                unit="TFLOP/s", frac=achieved / p_fp32, traffic=traffic,
                traffic_unit="DRAM bytes per step (ncu, profiles/ls_prop_kernel_dram_n5000.txt)",
                algorithmic_bytes=3.0 * 4 * D * float(N) * N,
                peak_basis="FP32 pipe 2 x 128 lanes x %d SMs x %.0f MHz (max SM clock, MEASURED_PEAKS.json)" % (nsm, sm_max),
                phase_ms={"forward": float(ph[0]), "backward": float(ph[1]), "decode": float(ph[2]),
                          "symmetrise": float(ph[3])})
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (2 * 128 * nsm * clocks["sm_mhz"] * 1e6 / 1e12)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=t_step, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic founder mosaics (seeded)",
                config={"workload": args.workload, "N": N, "L": L, "D": D, "decode_loci": "evenly spaced",
                        "prior": "uniform", "mu": w["mu"], "l2": "flushed before every timed step (256 MiB write)",
                        "parallelism": "replica per GPU" if world > 1 else "single GPU"},
                roofline=roof, clocks=clocks, gpu_launches=launches, pac=pac)

    # end to end through the C ABI with host buffers: pack from pinned host haplotypes, parameters,
    # run_all into a pinned host d, read back; copies inside the timed region
    if not args.no_e2e:
        h_pin = torch.from_numpy(np.ascontiguousarray(w["h"])).pin_memory().numpy()
        d_host = torch.empty((D, N, N), dtype=torch.float32, pin_memory=True).numpy()
        e2e_t, e2e_ph = [], []
        for s in range(1 + min(args.steps, 3)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = ls.ls_create(h_pin)            # the calls are synchronous: the phase times add up
            t1 = time.perf_counter()
            ls.ls_set_params(c2, w["rho"], w["mu"])
            t2 = time.perf_counter()
            ls.ls_run_all(c2, loci, d_host, want_pac=True)
            t3 = time.perf_counter()
            ls.ls_destroy(c2)
            torch.cuda.synchronize()
            t4 = time.perf_counter()
            if s > 0:
                e2e_t.append(t4 - t0)
                e2e_ph.append((t1 - t0, t2 - t1, t3 - t2, t4 - t3))
        te = max_over_ranks(float(np.mean(e2e_t)), world)
        ph = np.mean(np.array(e2e_ph), axis=0) * 1e3
        # the host link on this machine: one pinned device-to-host copy of d's size (outside the timed region)
        d_host_t = torch.from_numpy(d_host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_host_t.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        d2h_gbs = d.numel() * 4 / (time.perf_counter() - t0) / 1e9
        h2d = int(w["h"].nbytes + 8 * (L - 1) + 8)
        d2h = int(d_host.nbytes + 8 * N + 4 * N)
        line["e2e"] = {"value": world * cells / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "s_per_step": te,
                       "phases_ms": {"create (H2D + pack)": float(ph[0]), "set_params": float(ph[1]),
                                     "run_all (device + D2H of d)": float(ph[2]), "destroy": float(ph[3])},
                       "d2h_gbs_of_this_host": d2h_gbs}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(w, args.cpu_seconds, threads=args.cpu_threads)
    ls.ls_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
