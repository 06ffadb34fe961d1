#!/usr/bin/env python
"""Throughput benchmark of the Chebyshev-BdG hot path on GB300.

One step is one self-consistency iteration (paragraph after Eq. 20) of the
disordered s-wave 128x128 open lattice (eps_i ~ U[-0.5, 0.5], seed 1001,
t = 1, mu = -0.5, U = 2, T = 0.01) with M = 1024 Chebyshev moments and all
16384 sites as start vectors: Gershgorin rescale, damped Fermi coefficients,
ceil(M/2) applications of H~ per start vector with fused moments, the FP64
fold into Delta_i and n_i, and the linear mix.

Unit: vector-steps/s, one vector-step = one start vector advanced by one
application of H~ in the doubled recursion (it yields two moments); a step
of this workload is 16384 * 512 vector-steps.  The headline runs the
recursion in FP32 with FP64 folds; the plain FP64 form is measured beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun) every rank runs an independent replica (weak scaling):
the method exchanges nothing between start vectors inside an iteration.
"""
from __future__ import annotations

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

METRIC = ("Chebyshev BdG steps/s (vectors×H-apps), FP32 vs FP64 at ≤1e-4 Δ error; HBM %")
UNIT = "vector-steps/s"
L, M, SEED = 128, 1024, 1001
# per vector element and step: the stencil's 6 FMAs and half of a site's 6 product FMAs (FMA = 2 flops)
FP64_FLOPS_PER_ELEMENT_STEP = 18.0


def kernel_source_digest(sources):
    """First 16 hex digits of the SHA-256 of the kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for src in sources:
        with open(os.path.join(ROOT, "paper_1007_1609_gb300/csrc", src), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(sources=("step.cu",), pattern="step_real_kernel_fp32_*.md"):
    """DRAM bytes per launch of a recursion kernel from the committed ncu
    summary, or None when the kernel source changed since those counters were
    taken."""
    import glob
    import re
    digest = kernel_source_digest(sources)
    for path in glob.glob(os.path.join(ROOT, "profiles", pattern)):
        text = open(path).read()
        m = re.search(r"traffic_bytes_per_launch:\s*(\d+)\s+kernel_source_sha256_16:\s*([0-9a-f]+)", text)
        if m and m.group(2) == digest:
            return int(m.group(1)), os.path.relpath(path, ROOT)
    return None, None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device="cpu"):
    """Max of a per-rank float over all ranks (the timing rule for N > 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(problem, target_s=12.0, max_sites=1024):
    """The FP64 oracle, as it stands, on a bounded sample of start sites of the
    same workload (all M moments per site).  Returns (record, sites, delta, n)."""
    import numpy as np
    from oracle import oracle as orc
    p = problem
    ol = orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing,
                     p.coupling, p.delta0)
    a = orc.rescale(ol)
    rng = np.random.default_rng(2024)
    threads = orc.num_threads()
    n = max(threads, 8)
    sites = rng.choice(p.N, size=n, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    d, nn = orc.order_parameter_sites(ol, a, p.T, p.M, 1 << 16, sites)
    t1 = time.perf_counter() - t0
    n2 = int(min(max_sites, max(n, round(n * target_s / max(t1, 1e-3) / threads) * threads)))
    if n2 > n:
        sites = rng.choice(p.N, size=n2, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        d, nn = orc.order_parameter_sites(ol, a, p.T, p.M, 1 << 16, sites)
        t1 = time.perf_counter() - t0
    units = sites.size * math.ceil(p.M / 2)
    rec = {"value": units / t1, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": (f"{sites.size} random start sites of the same 128x128 lattice, all {p.M} "
                      f"moments each, folded to Delta_i and n_i ({t1:.1f} s; the oracle applies "
                      f"H~ {p.M - 1} times per site without doubling; value counts the doubled "
                      f"recursion's {math.ceil(p.M / 2)} vector-steps per site)")}
    return rec, sites, d, nn, a


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1007_1609_gb300 import workloads as wl
    from oracle import oracle as orc
    import numpy as np
    p = wl.swave_disordered(L, M, seed=SEED)
    ol = orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing,
                     p.coupling, p.delta0)
    threads = orc.num_threads()
    n_sites = max(threads, 16)
    rng = np.random.default_rng(99)
    times = []
    for k in range(args.warmup + args.steps):
        sites = rng.choice(p.N, size=n_sites, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        a = orc.rescale(ol)
        orc.order_parameter_sites(ol, a, p.T, p.M, 1 << 16, sites)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    t = sum(times)
    units = n_sites * math.ceil(p.M / 2) * len(times)
    value = units / t
    sample = (f"per step {n_sites} random start sites of the 128x128 disordered lattice, all "
              f"{p.M} moments each, folded to Delta_i and n_i (FP64 oracle, direct recursion)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "s-wave disordered 128x128 open, W=1.0 seed 1001, M=1024",
                   "start_vectors_per_step": n_sites},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1007_1609_gb300 import build as B
    B.build()
    from paper_1007_1609_gb300 import cbdg
    from paper_1007_1609_gb300 import workloads as wl

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    p = wl.swave_disordered(args.lattice, args.moments, seed=SEED)
    units_per_step = p.N * math.ceil(p.M / 2)
    stream = torch.cuda.Stream(device=dev)

    # ---------------- device-resident headline: FP32 recursion, FP64 folds
    lat = cbdg.Lattice(p, precision="fp32", stream=stream)
    if args.temporal is not None:
        lat.set_option(cbdg.CBDG_OPT_TEMPORAL_STEPS, args.temporal)
    for _ in range(args.warmup):
        lat.scf_step(p.T, p.M, p.mix)
    # the production path: every iteration after the second is a CUDA-graph replay
    cbdg.cbdg_launch_count(lat.handle, reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        diffs = [lat.scf_step(p.T, p.M, p.mix) for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, dev)
    launches = cbdg.cbdg_launch_count(lat.handle)
    value = world * units_per_step * args.steps / (ms_max / 1e3)
    # a separate profiled pass (direct launches, a CUDA event pair around every
    # recursion launch on the lattice's stream) gives the kernel's average
    # launch time for the roofline
    prof_iters = max(1, min(2, args.steps))
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_PROFILE, 1)
    cbdg.cbdg_profile_read(lat.handle, reset=True)
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(prof_iters):
        lat.scf_step(p.T, p.M, p.mix)
    pe1.record(stream)
    torch.cuda.synchronize()
    prof_ms = pe0.elapsed_time(pe1)
    step_ms, step_n, step_bytes = cbdg.cbdg_profile_read(lat.handle)
    k_used = cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_PROFILE, 0)

    # ---------------- end to end through the C ABI with host buffers
    host_delta = torch.from_numpy(np.ascontiguousarray(p.delta0)).pin_memory()
    host_out = torch.empty_like(host_delta).pin_memory()
    e2e_value = None
    if not args.no_e2e:
        lat_e = cbdg.Lattice(p, precision="fp32", stream=stream)
        if args.temporal is not None:
            lat_e.set_option(cbdg.CBDG_OPT_TEMPORAL_STEPS, args.temporal)
        for _ in range(1):
            cbdg.cbdg_set_delta(lat_e.handle, host_delta)
            cbdg.cbdg_scf_step(lat_e.handle, p.T, p.M, p.mix)
            cbdg.cbdg_get_delta(lat_e.handle, host_out)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            cbdg.cbdg_set_delta(lat_e.handle, host_delta)
            cbdg.cbdg_scf_step(lat_e.handle, p.T, p.M, p.mix)
            cbdg.cbdg_get_delta(lat_e.handle, host_out)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        lat_e.close()
        e2e_value = world * units_per_step * args.steps / e2e_s

    line = None
    if rank == 0:
        hbm, peak_kind = peaks()
        achieved = (step_bytes / step_n) / (step_ms / step_n / 1e3) / 1e9 if step_n else None
        if k_used >= 2:
            traffic, traffic_src = recorded_traffic(("step_multi.cu", "multi_pass.cuh"), "step_multi_kernel_fp32_*.md")
            kernel = (f"step_multi_kernel: FP32, {k_used} recursion steps per pass over the vectors "
                      "(reads j_(n-1), j_n; writes the last two), moment products fused; the "
                      "leftover step of each iteration runs step_real_kernel")
            if k_used == 3 and p.Lx > 64:
                kernel += ("; lean pass: level 0 read from its shared-memory ring, parameters in a ring "
                           "of their own, FP32 column sums")
        else:
            traffic, traffic_src = recorded_traffic()
            kernel = "step_real_kernel: FP32 recursion step with fused moment products"
        if args.lattice != L or args.moments != M:
            traffic, traffic_src = None, None  # recorded for the 128x128, M=1024 launch only
        vec_bytes = 2 * p.N * p.N * 4  # one FP32 block of all start vectors
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                    "traffic_source": traffic_src,
                    "kernel": kernel, "steps_per_pass": int(k_used),
                    "peak_kind": f"{peak_kind} (copy bandwidth)",
                    "algorithmic_bytes_per_launch": (4 if k_used >= 2 else 3) * vec_bytes,
                    "recursion_launches_per_step": step_n / prof_iters,
                    # the same time against the roofline of one step per pass (3 streams per step):
                    # what several steps per pass buy over the unfused recursion
                    "one_step_roofline_frac": ((3.0 * vec_bytes * k_used) / (step_ms / step_n / 1e3) / 1e9 / hbm
                                               if step_n and k_used >= 2 else None),
                    "avg_launch_ms": step_ms / step_n if step_n else None,
                    "avg_launch_source": (f"separate profiled pass of {prof_iters} iteration(s) after the timed "
                                          "region: CUDA events around every recursion launch on its stream"),
                    "share_of_step": step_ms / prof_ms if prof_ms else None}
        extra = {}
        ap = arith_peaks(cbdg, torch, stream, local)
        extra["arith_peaks"] = ap
        if not args.no_fp64:
            extra["fp64"] = fp64_leg(p, stream, cbdg, torch, units_per_step, fp64_peak=ap["fp64_fma"]["tflops"])
            extra["fp32_vs_fp64"] = {"speedup": value / world / extra["fp64"]["value"]}
        if not args.no_converge and args.lattice == L and args.moments == M:
            extra["converge"] = leg_converge(cbdg, wl, torch, stream, from_scratch=False)
        if not args.no_extras:
            extra["other_stages"] = extra_legs(cbdg, wl, torch, stream, hbm)
        cpu = None
        if not args.no_cpu_baseline:
            cpu, sites, od, on, oa = cpu_baseline(p)
            # accuracy of both GPU forms against the oracle on the sampled sites
            errs = {}
            for prec in ("fp32", "fp64"):
                lt = cbdg.Lattice(p, precision=prec, stream=stream)
                d, n = lt.order_parameter(p.T, p.M)
                errs[prec] = {"max_abs_delta_err": float(np.max(np.abs(d[sites] - od))),
                              "max_abs_n_err": float(np.max(np.abs(n[sites] - on))),
                              "sites": int(sites.size)}
                lt.close()
            extra["accuracy_vs_oracle_first_iteration"] = errs
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"s-wave disordered {p.Lx}x{p.Ly} open lattice, W=1.0 (seed 1001), "
                                   f"t=1, mu=-0.5, U=2, T=0.01, M={p.M}, all {p.N} sites as "
                                   "start vectors, FP32 recursion with FP64 folds",
                       "step": "one self-consistency iteration",
                       "units_per_step": units_per_step,
                       "l2": "no flush: the two recursion vectors are 2 x 2.1 GB per rank, "
                             "far larger than the 126 MB L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": None if e2e_value is None else {
                "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(host_delta.numel() * 16),
                "d2h_bytes_per_step": int(host_out.numel() * 16 + 8)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "scf_max_abs_ddelta": diffs[-1],
        }
        line.update(extra)
        # short copies of the FP64 comparison inside config (kept by line parsers that keep only
        # the contract's keys)
        if "fp64" in extra:
            line["config"]["fp64_vector_steps_per_s"] = extra["fp64"]["value"]
            line["config"]["fp32_vs_fp64_speedup"] = extra["fp32_vs_fp64"]["speedup"]
        if "converge" in extra:
            line["config"]["converged_max_abs_delta_fp32_vs_fp64"] = extra["converge"]["max_abs_delta_fp32_vs_fp64"]
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def leg_contraction(cbdg, torch, stream, shape=(65536, 2048, 512), tf32_peak=None):
    """LDOS contraction on the tensor cores at the vortex-lattice shape:
    [65536 sites x 2048 moments] . [2048 x 512 energies], 3xTF32.  Times the
    tcgen05 kernel on pre-split operand planes (the roofline) and the whole
    call that also splits both FP32 operands."""
    m, k, n = shape
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn((m, k), generator=g, device="cuda", dtype=torch.float32)
    B = torch.randn((n, k), generator=g, device="cuda", dtype=torch.float32)
    D = torch.empty((m, n), device="cuda", dtype=torch.float32)
    kp = cbdg.cbdg_contract_kp(k)
    ahi, alo = (torch.empty((m, kp), device="cuda", dtype=torch.float32) for _ in range(2))
    bhi, blo = (torch.empty((n, kp), device="cuda", dtype=torch.float32) for _ in range(2))
    cbdg.cbdg_split_tf32(A, k, m, k, ahi, alo, stream)
    cbdg.cbdg_split_tf32(B, k, n, k, bhi, blo, stream)
    flops = 3 * 2.0 * m * n * k
    reps = 5

    def timed(fn):
        fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_kernel = timed(lambda: cbdg.cbdg_contract_tf32x3_planes(ahi, alo, bhi, blo, kp, D, n, m, n, stream))
    ms_call = timed(lambda: cbdg.cbdg_contract_tf32x3(A, k, B, k, D, n, m, n, k, stream))
    tflops = flops / (ms_kernel * 1e-3) / 1e12
    if tf32_peak:
        peak, peak_kind = tf32_peak, "measured (cbdg_measure_peak, tcgen05 kind::tf32 at the kernel's MMA shape)"
    else:
        peak, peak_kind = bf16_peak() * 0.5, "measured bf16 dense burst x 0.5 (nominal tf32/bf16 ratio)"
    useful = 2.0 * m * n * k
    return {"shape": [m, k, n], "ms": ms_kernel, "tflops": tflops,
            "useful_tflops": useful / (ms_kernel * 1e-3) / 1e12,
            "call_ms_with_split": ms_call, "call_tflops_with_split": flops / (ms_call * 1e-3) / 1e12,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "peak_kind": peak_kind,
                         "note": "contract_kernel alone; achieved counts the 3 TF32 products per term "
                                 "(hi*hi + hi*lo + lo*hi) the tensor cores execute; useful_tflops counts "
                                 "the method's 2 m n k"}}


def leg_dwave(cbdg, wl, stream, hbm, columns=4096):
    """General recursion step (complex64, t', bond pairing, Peierls field) on
    the 256x256 vortex lattice, a chunk of `columns` start sites."""
    import numpy as np
    pv = wl.dwave_vortex(256, 34)
    lat = cbdg.Lattice(pv, precision="fp32", stream=stream, complex_field=True)
    sites = (np.arange(columns, dtype=np.int64) * (pv.N // columns)).astype(np.int32)
    lat.moments(sites, 8)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_PROFILE, 1)
    cbdg.cbdg_profile_read(lat.handle, reset=True)
    lat.moments(sites, pv.M)
    sms, sn, sb = cbdg.cbdg_profile_read(lat.handle)
    tile = lat.last_tile()
    lat.close()
    return {"lattice": "256x256 periodic, t'=-0.3, 2 h/2e flux, bond pairing, complex64",
            "columns": int(columns), "launches": sn, "avg_launch_ms": sms / sn, "tile": list(tile),
            "roofline": {"bound": "hbm", "achieved": sb / (sms * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": sb / (sms * 1e-3) / 1e9 / hbm}}


def leg_ensemble(cbdg, wl, stream, samples=256):
    """256 disordered lattices (sides 32..96, M = 512): one graph-replayed
    self-consistency iteration (fewer samples for profiling runs)."""
    probs = wl.ensemble()[:samples]
    ens = cbdg.Ensemble(probs, stream=stream)
    t0 = time.perf_counter()
    ens.scf(0.01, 512, 0.5, 0.0, 1)  # includes the graph capture
    t1 = time.perf_counter()
    ens.scf(0.01, 512, 0.5, 0.0, 1)
    t2 = time.perf_counter()
    ens.close()
    units = sum(p.N for p in probs) * 256
    # 255 doubled steps per column: three-step passes (4 vector streams of 2N x 4 B each)
    # while three remain, then single steps (3 streams)
    steps = (512 + 1) // 2 - 1
    streams = 4 * (steps // 3) + 3 * (steps % 3)
    algo_bytes = sum(streams * 2 * p.N * 4 * p.N for p in probs)
    return {"samples": len(probs), "s_per_iteration": t2 - t1, "first_call_s": t1 - t0,
            "vector_steps_per_s": units / (t2 - t1), "algorithmic_gbs": algo_bytes / (t2 - t1) / 1e9,
            "algorithmic_bytes": algo_bytes, "streams_per_column": streams,
            "streams_per_column_one_step_per_pass": 3 * steps}


def adjoint_streams(M, multi=False):
    """Vector streams (reads + writes of one 2N x B vector) of one adjoint run
    as the library schedules it: forward with checkpoints every S = ceil(sqrt M)
    steps, per segment the checkpoint copies and the recomputation, the
    reverse recursion (3 streams per step) and the gradient accumulation
    (lambda_m and j_(m-1): 2 streams per moment).  multi: the forward,
    recomputed and reverse recursions run three steps per pass where three
    remain in the segment (else two, else one): in place a pass moves 4
    vectors, with every level written 2 + K."""
    import math
    S = max(2, math.ceil(math.sqrt(M)))
    nseg = (M + S - 1) // S

    def run(n, to, out_of_place):
        s = 0
        while n < to:
            k = 3 if multi and to - n >= 3 else (2 if multi and to - n >= 2 else 1)
            s += (2 + k if out_of_place else 4) if k > 1 else 3
            n += k
        return s
    fwd, n = 2 * 2, 1  # copies of j_0, j_1 into checkpoint 0
    for k in range(1, nseg):
        to = k * S + 1 if k * S + 1 < M else k * S
        fwd += run(n, to, False) + 2 * (2 if to == k * S + 1 else 1)
        n = to
    rec, rev, m = 0, 0, M
    for k in reversed(range(nseg)):
        r_end = min(S, M - k * S)
        rec += 2 + (2 if r_end > 1 else 0) + run(1, max(1, r_end - 1), True)
        # lam_(m-1) .. lam_(kS+1), every level written (the first, lam_(M-1), is its source alone)
        if m == M:
            m = M - 1
        rev += run(k * S + 1, m, True)
        m = k * S + 1
    rev += 2 * (M - 1)  # accumulation: lam_m and j_(m-1) for m = M-1 .. 1
    return fwd + rec + rev


def leg_adjoint(cbdg, wl, stream, hbm):
    """Gradient of one self-consistency map, 64x64, M = 512 (FP64 and FP32),
    with the algorithmic bytes of the implemented schedule (adjoint_streams);
    and of the general-lattice map (64x64 periodic d-wave lattice with field,
    t' and two vortices: complex64 vectors, one step per launch), FP32."""
    import numpy as np
    out = {}
    pc = wl.currents_dwave(64, 512)
    lc = cbdg.Lattice(pc, precision="fp32", complex_field=True, stream=stream)
    lc.order_parameter(pc.T, pc.M)
    gc = (np.random.default_rng(1).normal(size=(pc.N, 4)) * (np.abs(pc.delta0) > 0)).astype(np.complex128)
    lc.backward(pc.T, pc.M, gc)
    t0 = time.perf_counter()
    lc.backward(pc.T, pc.M, gc)
    dt = time.perf_counter() - t0
    lc.close()
    vb = 2 * pc.N * pc.N * 8
    gbs = adjoint_streams(pc.M) * vb / dt / 1e9
    out["general_fp32_s"] = dt
    out["general_fp32_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                    "streams": adjoint_streams(pc.M), "vector_bytes": vb,
                                    "note": "64x64 d-wave vortex lattice (bond pairing, t', field), complex64; "
                                            "whole backward call over its algorithmic bytes"}
    pg = wl.gradient_case()
    for prec, es in (("fp64", 8), ("fp32", 4)):
        lg = cbdg.Lattice(pg, precision=prec, stream=stream)
        d, _ = lg.order_parameter(pg.T, pg.M)
        w = (2.0 * (d.real - pg.extra["target"])).astype(np.complex128)
        lg.backward(pg.T, pg.M, w)
        t0 = time.perf_counter()
        lg.backward(pg.T, pg.M, w)
        dt = time.perf_counter() - t0
        out[f"{prec}_s"] = dt
        lg.close()
        if prec == "fp32":
            vb = 2 * pg.N * pg.N * es
            streams = adjoint_streams(pg.M, multi=True)
            gbs = streams * vb / dt / 1e9
            out["fp32_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                    "frac": gbs / hbm, "streams": streams, "vector_bytes": vb,
                                    "streams_one_step_per_pass": adjoint_streams(pg.M),
                                    "note": "whole backward call (forward with checkpoints, recomputation and "
                                            "reverse recursion three steps per pass, accumulation) over its "
                                            "algorithmic bytes"}
    return out


def leg_tiny(cbdg, wl, stream):
    """The 16x16 clean lattice (M = 256, all 256 sites): 10 mixed
    self-consistency iterations from uniform Delta = 0.5, replayed as CUDA
    graphs.  The whole recursion runs in shared memory (one launch per
    iteration); "*_streamed" is the same with the HBM-streaming kernels."""
    p = wl.swave_clean(16, 256)
    out = {}
    for prec, resident in (("fp64", 1), ("fp32", 1), ("fp64", 0), ("fp32", 0)):
        lat = cbdg.Lattice(p, precision=prec, stream=stream)
        lat.set_option(cbdg.CBDG_OPT_RESIDENT, resident)
        lat.scf_step(p.T, p.M, p.mix)  # warm-up (tables, buffers)
        lat.delta = p.delta0
        t0 = time.perf_counter()
        for _ in range(10):
            diff = lat.scf_step(p.T, p.M, p.mix)
        dt = time.perf_counter() - t0
        out[prec if resident else prec + "_streamed"] = {
            "ms_10_iterations": dt * 1e3, "ms_per_iteration": dt * 1e2,
            "vector_steps_per_s": 10 * p.N * ((p.M + 1) // 2) / dt, "last_max_abs_ddelta": diff}
        lat.close()
    return out


def leg_currents(cbdg, wl, torch, stream, hbm):
    """Bond currents (Eq. 20) on the vortex-imprinted d-wave lattice, 128x128,
    M = 512, FP32 complex vectors: all 16384 sites as start vectors, 510
    direct recursion steps each plus the nearest-bond readout.  Event-timed
    whole call and per-step kernel time (CBDG_OPT_PROFILE)."""
    p = wl.currents_dwave(128, 512)
    lat = cbdg.Lattice(p, precision="fp32", stream=stream)
    lat.bond_currents(p.T, 8)  # buffers and tables
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_PROFILE, 1)
    cbdg.cbdg_profile_read(lat.handle, reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    J = lat.bond_currents(p.T, p.M)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sms, sn, sb = cbdg.cbdg_profile_read(lat.handle)
    tile = lat.last_tile()
    lat.close()
    units = p.N * (p.M - 2)
    return {"lattice": "128x128 periodic, t'=-0.3, 2 h/2e flux, 2 imprinted vortices, bond pairing, complex64",
            "M": p.M, "call_ms": ms, "vector_steps_per_s": units / (ms * 1e-3),
            "step_launches": sn, "avg_step_ms": sms / max(sn, 1), "step_share_of_call": sms / ms,
            "tile": list(tile), "max_abs_J": float(abs(J).max()),
            "roofline": {"bound": "hbm", "achieved": sb / (sms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": sb / (sms * 1e-3) / 1e9 / hbm,
                         "note": "step_cplx_kernel (direct mode), 3 vector streams of 2N x N x 8 B per step"}}


def leg_junction(cbdg, wl, torch, stream, hbm):
    """The S/N slab after the paper's first example (a 500-site periodic
    plane x 320 layers, U = 0 on the top 20 layers, M = 2048, FP32): one
    self-consistency iteration (second call, graph replay) with one start
    site per layer (the plane's translations, cbdg_set_symmetry), and the
    surface LDOS (64 surface sites x 201 energies) with the Lorentz kernel at
    a broadening of 0.001 t."""
    import numpy as np
    p = wl.sn_slab()
    lat = cbdg.Lattice(p, precision="fp32", stream=stream)
    lat.set_coupling(p.extra["coupling_site"])
    lat.set_symmetry(p.extra["symmetry"])
    lat.scf_step(p.T, p.M, p.mix)
    t0 = time.perf_counter()
    diff = lat.scf_step(p.T, p.M, p.mix)
    t1 = time.perf_counter()
    lam = lat.lorentz_lambda(p.extra["broadening"], p.M)
    E = p.extra["energy_frac"] * lat.rescale
    sites = p.extra["surface_sites"][:64]
    lat.ldos(sites, p.M, E, kernel="lorentz", lam=lam)
    t2 = time.perf_counter()
    rho = lat.ldos(sites, p.M, E, kernel="lorentz", lam=lam)
    t3 = time.perf_counter()
    d = lat.delta
    # recursion kernels alone (profiled iteration: direct launches, no graph)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_PROFILE, 1)
    cbdg.cbdg_profile_read(lat.handle, reset=True)
    lat.order_parameter(p.T, p.M)
    sms, sn, sb = cbdg.cbdg_profile_read(lat.handle)
    k = cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL)
    tile = lat.last_tile()
    lat.close()
    L = p.Lx
    units = p.Ly * ((p.M + 1) // 2)
    return {"lattice": f"{L}x{p.Ly}, periodic x (the plane), open y, S rows 0-299 (U = 1.41), N rows 300-319 (U = 0)",
            "M": p.M, "start_vectors": int(p.Ly), "scf_iteration_s": t1 - t0, "vector_steps_per_s": units / (t1 - t0),
            "max_abs_ddelta": diff, "delta_bulk": float(abs(d[L * 150])), "delta_interface": float(abs(d[L * 299])),
            "surface_ldos_s": t3 - t2, "lorentz_lambda": lam, "surface_ldos_at_0": float(rho[:, 100].mean()),
            "steps_per_pass": k, "tile": list(tile), "recursion_launches": sn, "recursion_ms": sms,
            "roofline": {"bound": "hbm", "achieved": sb / (sms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": sb / (sms * 1e-3) / 1e9 / hbm,
                         "note": "recursion kernels over their algorithmic bytes (one start site per layer)"}}


def leg_green(cbdg, wl, torch, stream, fp64_peak=None):
    """Nonlocal Green's functions (gf1) around a vortex core of the 128x128
    d-wave lattice, M = 1024: 16 start sites (a 4x4 block at the core) x 256
    targets (a 16x16 block) x 512 energies in [-0.5a, 0.5a], device outputs.
    The recursion (16 columns, 1022 steps) is timed by cbdg_green_moments;
    the FP64 contraction is the difference to cbdg_green_function (weights
    and two [M] x [M x 512] complex contractions per (site, target))."""
    import numpy as np
    p = wl.currents_dwave(128, 1024)
    L, M, n_E = 128, p.M, 512
    lat = cbdg.Lattice(p, precision="fp32", stream=stream)
    xs, ys = np.meshgrid(np.arange(30, 34), np.arange(30, 34))
    sites = (xs + L * ys).ravel().astype(np.int32)
    xt, yt = np.meshgrid(np.arange(24, 40), np.arange(24, 40))
    targets = (xt + L * yt).ravel().astype(np.int32)
    ns, nt = sites.size, targets.size
    lat.green_moments(sites[:1], targets[:1], 8)   # buffers; sets the rescale
    E = np.linspace(-0.5, 0.5, n_E) * lat.rescale
    a11 = torch.empty((ns, M, nt), dtype=torch.complex128, device="cuda")
    a12 = torch.empty_like(a11)
    G11 = torch.empty((ns, nt, n_E), dtype=torch.complex128, device="cuda")
    G12 = torch.empty_like(G11)
    dE = torch.from_numpy(E).cuda()

    def moments():
        cbdg.cbdg_green_moments(lat.handle, sites, ns, targets, nt, M, a11, a12)

    def green():
        cbdg.cbdg_green_function(lat.handle, sites, ns, targets, nt, M, 0, 0.0, dE, n_E, G11, G12)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    t_mom = timed(moments)
    t_all = timed(green)
    lat.close()
    flops = 2 * 8.0 * ns * nt * M * n_E
    t_con = max(t_all - t_mom, 1e-9)
    tf = flops / t_con / 1e12
    return {"lattice": "128x128 d-wave vortex lattice, complex64 recursion", "M": M, "sites": ns, "targets": nt,
            "energies": n_E, "moments_s": t_mom, "green_function_s": t_all, "contraction_s": t_con,
            "roofline": {"bound": "alu", "achieved": tf, "peak": fp64_peak or 1.25, "unit": "TFLOP/s",
                         "frac": tf / (fp64_peak or 1.25),
                         "peak_kind": ("measured (cbdg_measure_peak, FP64 FMA)" if fp64_peak
                                       else "nominal FP64 rate of the profiling recipe's table"),
                         "note": "green_contract_kernel, FP64 complex multiply-adds (8 flops each), from the call "
                                 "time difference"}}


def scf_to(lat, p, tol, max_iter, torch, err_tol=None):
    """Self-consistency iterations (linear mixing p.mix) until max|Delta_out -
    Delta| < tol or, with err_tol, until the estimated distance of the mixed
    Delta to the fixed point is below err_tol: near the fixed point the
    mixed iteration contracts by rho = r_k / r_(k-1) per step and leaves
    Delta_(k+1) - Delta* = rho (Delta_k - Delta*) with |Delta_k - Delta*| =
    r_k / (1 - F') = mix r_k / (1 - rho), i.e. an error of
    rho mix r_k / (1 - rho).  Returns (iterations, seconds, last max|dDelta|,
    last error estimate or None)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, diff, prev, est = 0, float("inf"), None, None
    while it < max_iter:
        diff = lat.scf_step(p.T, p.M, p.mix)
        it += 1
        if err_tol is not None and prev is not None and 0.0 < diff < prev:
            rho = diff / prev
            est = rho * p.mix * diff / (1.0 - rho)
            if est < err_tol:
                break
        elif err_tol is None and diff < tol:
            break
        prev = diff
    torch.cuda.synchronize()
    return it, time.perf_counter() - t0, diff, est


def leg_converge(cbdg, wl, torch, stream, from_scratch=True, tol32=1e-4, tol64=1e-6, max_iter=400,
                 margin=0.5):
    """The 128x128 disordered workload to self-consistency in both forms: the
    FP32 recursion (FP64 folds and mixing) from Delta = 0.5, stopped once the
    estimated distance to the fixed point is below margin x 1e-4 (scf_to), and the
    plain FP64 form to max|dDelta| < 1e-6, from Delta = 0.5 (time to
    solution) or, when from_scratch is False, from the FP32 solution.
    Reports iterations, times and max_i |Delta_FP32 - Delta_FP64| over all
    sites; with from_scratch also the FP32 result at the update tolerance
    max|dDelta| < 1e-4 alone."""
    import numpy as np
    p = wl.swave_disordered(L, M, seed=SEED)
    out = {"sites": int(p.N)}
    d32_upd = None
    if from_scratch:
        lat = cbdg.Lattice(p, precision="fp32", stream=stream)
        n, t, r, _ = scf_to(lat, p, tol32, max_iter, torch)
        d32_upd = lat.delta
        lat.close()
        out["fp32_update_tol"] = {"iterations": n, "seconds": t, "last_max_abs_ddelta": r, "tol": tol32}
    lat32 = cbdg.Lattice(p, precision="fp32", stream=stream)
    n32, t32, r32, e32 = scf_to(lat32, p, None, max_iter, torch, err_tol=margin * tol32)
    d32 = lat32.delta
    lat32.close()
    out["fp32"] = {"iterations": n32, "seconds": t32, "last_max_abs_ddelta": r32, "estimated_error": e32,
                   "stop": f"estimated |Delta - Delta*| < {margin * tol32:g} (target {tol32:g})"}
    lat64 = cbdg.Lattice(p, precision="fp64", stream=stream)
    if not from_scratch:
        lat64.delta = d32
    n64, t64, r64, _ = scf_to(lat64, p, tol64, max_iter, torch)
    d64 = lat64.delta
    lat64.close()
    key = "fp64" if from_scratch else "fp64_from_fp32_solution"
    out[key] = {"iterations": n64, "seconds": t64, "last_max_abs_ddelta": r64, "tol": tol64}
    err = np.abs(d32 - d64)
    out["max_abs_delta_fp32_vs_fp64"] = float(err.max())
    out["mean_abs_delta_fp32_vs_fp64"] = float(err.mean())
    if d32_upd is not None:
        out["fp32_update_tol"]["max_abs_delta_vs_fp64"] = float(np.abs(d32_upd - d64).max())
    out["delta_fp64_range"] = [float(np.abs(d64).min()), float(np.abs(d64).max())]
    if from_scratch:
        out["time_to_solution_speedup"] = t64 / t32
    return out


def extra_legs(cbdg, wl, torch, stream, hbm, only=None, columns=4096, samples=256):
    """Other hot-path stages at their workload sizes (not the headline)."""
    ap = arith_peaks(cbdg, torch, stream)
    legs = {
        "tiny": lambda: leg_tiny(cbdg, wl, stream),
        "contraction": lambda: leg_contraction(cbdg, torch, stream, tf32_peak=ap["tf32_mma"]["tflops"]),
        "dwave": lambda: leg_dwave(cbdg, wl, stream, hbm, columns),
        "ensemble": lambda: leg_ensemble(cbdg, wl, stream, samples),
        "adjoint": lambda: leg_adjoint(cbdg, wl, stream, hbm),
        "currents": lambda: leg_currents(cbdg, wl, torch, stream, hbm),
        "junction": lambda: leg_junction(cbdg, wl, torch, stream, hbm),
        "green": lambda: leg_green(cbdg, wl, torch, stream, fp64_peak=ap["fp64_fma"]["tflops"]),
    }
    if only == "peaks":
        return {"peaks": ap}
    if only == "converge":
        return {"converge": leg_converge(cbdg, wl, torch, stream)}
    return {name: fn() for name, fn in legs.items() if only is None or only == name}


_ARITH = {}


def arith_peaks(cbdg, torch, stream, local=0):
    """FP64 / FP32 FMA and tcgen05 kind::tf32 MMA peaks of this GPU from the
    library's own probes (cbdg_measure_peak): one warm-up and one CUDA-event
    timed launch each (about 0.1 s), SM clocks sampled meanwhile.  Cached per
    process.  TFLOP/s."""
    if _ARITH:
        return _ARITH
    specs = (("fp64_fma", cbdg.CBDG_PEAK_FP64_FMA, 30000),
             ("fp32_fma", cbdg.CBDG_PEAK_FP32_FMA, 750000),
             ("tf32_mma", cbdg.CBDG_PEAK_TF32_MMA, 1 << 20))
    out = {}
    with ClockSampler(local) as clk:
        for name, kind, work in specs:
            cbdg.cbdg_measure_peak(kind, max(1, work // 16), stream)
            cbdg.cbdg_peak_status(stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = cbdg.cbdg_measure_peak(kind, work, stream)
            e1.record(stream)
            cbdg.cbdg_peak_status(stream)
            ms = e0.elapsed_time(e1)
            out[name] = {"tflops": flops / (ms * 1e-3) / 1e12, "ms": ms, "flops": flops}
    out["clocks"] = clk.summary()
    out["how"] = ("cbdg_measure_peak: FP64/FP32 -- 8/16 independent FMA chains per thread, 8 CTAs x 256 threads "
                  "per SM; TF32 -- tcgen05.mma kind::tf32 M=128 N=256 K=8 from shared memory into tensor "
                  "memory, one CTA per SM; one CUDA-event timed launch each after a warm-up")
    _ARITH.update(out)
    return _ARITH


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def fp64_leg(p, stream, cbdg, torch, units_per_step, fp64_peak=None):
    """The plain FP64 form on the same GPU: one warm-up and one timed iteration."""
    lat = cbdg.Lattice(p, precision="fp64", stream=stream)
    lat.scf_step(p.T, p.M, p.mix)
    lat.delta = p.delta0
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_PROFILE, 1)
    cbdg.cbdg_profile_read(lat.handle, reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.scf_step(p.T, p.M, p.mix)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    step_ms, step_n, step_bytes = cbdg.cbdg_profile_read(lat.handle)
    lat.close()
    elements = 2 * p.N * p.N  # rows x columns advanced per launch
    flops = FP64_FLOPS_PER_ELEMENT_STEP * elements * step_n
    return {"value": units_per_step / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "dtype": "f64",
            "roofline": {"bound": "alu", "achieved": flops / (step_ms / 1e3) / 1e12,
                         "peak": fp64_peak or 1.25, "unit": "TFLOP/s",
                         "frac": flops / (step_ms / 1e3) / 1e12 / (fp64_peak or 1.25),
                         "peak_kind": ("measured (cbdg_measure_peak, FP64 FMA)" if fp64_peak
                                       else "nominal FP64 rate of the profiling recipe's table"),
                         "hbm_gbs": step_bytes / (step_ms / 1e3) / 1e9}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-converge", action="store_true",
                    help="skip the FP32-vs-FP64 self-consistency comparison (about 90 s)")
    ap.add_argument("--stage", default=None, choices=["tiny", "contraction", "dwave", "ensemble", "adjoint", "currents", "junction", "green",
                             "converge", "peaks"],
                    help="measure only this stage and print its record (profiling runs)")
    ap.add_argument("--lattice", type=int, default=L,
                    help="lattice side (profiling of smaller cases; the metric is quoted at 128)")
    ap.add_argument("--moments", type=int, default=M)
    ap.add_argument("--samples", type=int, default=256,
                    help="lattices of the ensemble stage (--stage ensemble)")
    ap.add_argument("--columns", type=int, default=4096,
                    help="start vectors of the d-wave stage (--stage dwave)")
    ap.add_argument("--temporal", type=int, default=None,
                    help="recursion steps per pass over the vectors (1..4; default: library choice)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.stage is not None:
        import torch
        from paper_1007_1609_gb300 import build as B
        B.build()
        from paper_1007_1609_gb300 import cbdg
        from paper_1007_1609_gb300 import workloads as wl
        stream = torch.cuda.Stream()
        hbm, _ = peaks()
        rec = extra_legs(cbdg, wl, torch, stream, hbm, only=args.stage, columns=args.columns,
                         samples=args.samples)
        print(json.dumps({"stage": args.stage, **rec}), flush=True)
        return 0
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
