#!/usr/bin/env python3
"""Benchmark: FMM evaluations per second (E, F, dV/dlambda) at 500k atoms.

One step = one full FMM evaluation (binning, P2M, M2M, FP64 root/lattice,
M2L, L2L, L2P + P2P, reductions) of the solvated 500,000-atom periodic system
(17 nm box, 160,000 three-site waters plus four 5,000-atom charged clusters
with 200 titratable sites; p = 10, depth 5), from unsorted positions in HBM
to E, F (input order) and dV/dlambda.  Synthetic, seeded inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|tf32|3xtf32|3xbf16|fp16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Under torchrun (N > 1) every rank evaluates its own replica of the system
(the path runs replicas only; there is no data-path collective), and rank 0
prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM evals/s (E, F, dV/dlambda) at 500k atoms, mixed vs FP32, rel err <= 1e-4"
WORKLOAD = "solvated_500k: periodic 17 nm cube, 500,000 atoms (160,000 waters + 4 x 5,000-atom clusters, 200 sites), p=10, depth 5"
L2_BYTES = 126 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "tf32", "3xtf32", "3xbf16", "fp16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--small", action="store_true", help="30k-atom system (for profiling runs)")
    ap.add_argument("--workload", default="solvated_500k", choices=["solvated_500k", "batch64", "loop1000"],
                    help="batch64: 64 uneven replicas in one graph; loop1000: lambda-dynamics loop")
    return ap.parse_args()


def aggregate_ms(pg, ms: float, device=None) -> float:
    """Max of a per-rank time over the process group (the job is as fast as its slowest rank);
    the whole-job throughput is then world_size * units / max_ms."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        out.update(sm_mhz=statistics.median(r[0] for r in rows), sm_max_mhz=max(r[1] for r in rows),
                   reasons=reasons, samples=len(rows))
        return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one M2L launch on this workload,
# from an ncu capture of the tensor-core kernel built from the source with this sha1; reported
# only while the source is unchanged.
NCU_M2L_TRAFFIC = {
    "sha1": "a765e9757b43773db31cea9c84dcc9b9bddeee1d",
    "fp16": 27_469_824 + 0,  # the launch of the two finest levels (256 tiles of at most 192 rows)
}


def m2l_traffic(precision):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2410_01626_b300", "csrc", "m2l_tc.cu")
    try:
        with open(src, "rb") as fh:
            sha = hashlib.sha1(fh.read()).hexdigest()
    except OSError:
        return None
    return NCU_M2L_TRAFFIC.get(precision) if sha == NCU_M2L_TRAFFIC["sha1"] else None


def step_stats(step_ms):
    """Median, 10th and 90th percentile (nearest rank) of this rank's per-step device times."""
    v = sorted(step_ms)
    pick = lambda q: v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]
    return {"median": statistics.median(v), "p10": pick(0.10), "p90": pick(0.90), "n": len(v)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ oracle timing
def oracle_sample_cost(sys_, targets, tol=1e-8, seed=0):
    """One FP64 Ewald oracle call on `targets` random atoms of the system.  Returns the wall
    seconds of its two phases from the oracle's own clock: the structure factors (the fixed
    cost of any evaluation, every atom's charge) and the per-target sums divided by `targets`."""
    import numpy as np
    import oracle
    n = len(sys_["qA"])
    t = np.random.default_rng(seed).choice(n, targets, replace=False)
    oracle.evaluate(sys_, targets=t, tol=tol, site_atoms=False)
    sf, tg = oracle.ewald_phase_seconds()
    return sf, tg / targets


def oracle_targets():
    """Targets per oracle sample: a multiple of the oracle's dynamic chunk (8) times its threads,
    so that every thread gets the same number of chunks."""
    import oracle
    return 64 * oracle.nthreads()


def time_oracle(sys_, tol=1e-8, repeats=2, check_full=None):
    """The cost of one full FP64 Ewald evaluation of all N atoms on the host cores, by the
    model fixed + N x per-target with both terms measured by the oracle's phase clock on a
    bounded sample (median of `repeats` samples of oracle_targets() random atoms).  With
    `check_full` (a smaller system), that system is also evaluated in full and its measured
    time is reported beside the model's prediction, as a check of the model."""
    import statistics
    import oracle
    n = len(sys_["qA"])
    T = oracle_targets()
    runs = [oracle_sample_cost(sys_, T, tol, seed=r) for r in range(repeats)]
    sf = statistics.median(r[0] for r in runs)
    per = statistics.median(r[1] for r in runs)
    full = sf + n * per
    out = {"value": 1.0 / full, "unit": "evals/s", "cores": oracle.nthreads(), "kind": "oracle",
           "extrapolated": True,
           "sample": (f"FP64 Ewald oracle (tol {tol:g}) on {T} random target atoms of the {n}-atom system, "
                      f"median of {repeats}; one full evaluation = structure factors {sf:.2f} s + "
                      f"{n} x {per * 1e3:.4f} ms per target = {full:.0f} s (extrapolated from the sample)"),
           "structure_factor_s": sf, "per_target_s": per, "full_eval_s_model": full}
    if check_full is not None:
        import time as _t
        m = len(check_full["qA"])
        runs_c = [oracle_sample_cost(check_full, T, tol, seed=99 + r) for r in range(repeats)]
        sf_c = statistics.median(r[0] for r in runs_c)
        per_c = statistics.median(r[1] for r in runs_c)
        a = _t.perf_counter()
        oracle.evaluate(check_full, tol=tol)  # every atom: a real full evaluation
        measured = _t.perf_counter() - a
        model = sf_c + m * per_c
        out["check_full"] = {"atoms": m, "measured_s": measured, "model_s": model, "model_over_measured": model / measured,
                             "note": "one full FP64 Ewald evaluation of every atom, timed, against the sample model"}
    return out


def run_reference(args):
    """The FP64 CPU oracle as the reference arm, on the same workload.  Each timed step is one
    bounded sample (oracle_targets() random target atoms with the full structure factors); its
    phase clock gives the step's estimate of one full evaluation of all N atoms (structure
    factors + N x per-target cost).  `value` is that extrapolated rate; `ms_per_step` is the
    sample's own measured wall time."""
    import statistics
    import oracle
    import synth
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    s = synth.solvated_30k() if args.small else synth.solvated_500k()
    n = len(s["qA"])
    T = oracle_targets()
    for w in range(args.warmup):
        oracle_sample_cost(s, T, seed=1000 + w)
    full, wall = [], []
    for i in range(args.steps):
        a = time.perf_counter()
        sf, per = oracle_sample_cost(s, T, seed=i)
        wall.append(time.perf_counter() - a)
        full.append(sf + n * per)
    est = statistics.median(full)
    val = 1.0 / est
    cpu = {"value": val, "unit": "evals/s", "cores": oracle.nthreads(), "kind": "oracle", "extrapolated": True,
           "sample": (f"each step: FP64 Ewald oracle (tol 1e-8) on {T} random target atoms of the {n}-atom system "
                      f"with the full structure factors; the step's phase clock gives one full evaluation as "
                      f"structure factors + N x per-target cost (median over steps {est:.0f} s, extrapolated)"),
           "full_eval_s_model": est}
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(wall) / len(wall),
            "value_is_extrapolated": True, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.small else "solvated_30k", "precision": "fp64"},
            "cpu_baseline": cpu,
            "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ native
def run_native(args):
    import numpy as np
    import torch

    import synth
    from paper_2410_01626_b300 import FMM

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    s = synth.solvated_30k(p=10) if args.small else synth.solvated_500k()
    if args.small:
        s["depth"] = 4
    n, K = len(s["qA"]), len(s["lam"])
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in ("x", "qA", "qB", "site", "lam")}

    from paper_2410_01626_b300.binding import load as _load
    precision = args.precision
    if precision == "auto":  # the FP16 tensor-core mode (split low degrees) when the library offers it for this p
        try:
            FMM(s["L"], True, s["p"], 0, precision="fp16").close()
            precision = "fp16"
        except Exception:
            precision = "fp32"

    def solver(prec):
        f = FMM(s["L"], True, s["p"], s["depth"], precision=prec)
        f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
        return f

    f = solver(precision)
    E, F, dV, _ = f.outputs(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one_step():
        f.eval_into(t["x"], E, F, dV)

    for _ in range(max(args.warmup, 3)):
        one_step()
    torch.cuda.synchronize()

    # per-stage device times on the eval stream (instrumented eval, outside the timed region)
    f.set_profiling(True)
    stage_runs = []
    for _ in range(3):
        flush.zero_()
        one_step()
        stage_runs.append(f.stage_times())
    f.set_profiling(False)
    stages = {k: statistics.median(r[k] for r in stage_runs) for k in stage_runs[0]}
    # the same with every stage run alone, one after the other: each kernel's own duration,
    # which its roofline needs (in the ordinary evaluation the stages share the SMs)
    f.set_profiling(True, serial=True)
    alone_runs = []
    for _ in range(3):
        flush.zero_()
        one_step()
        alone_runs.append(f.stage_times())
    f.set_profiling(False)
    stages_alone = {k: statistics.median(r[k] for r in alone_runs) for k in alone_runs[0]}
    # leaving profiling mode drops the handle's evaluation graph: warm up again, so that its
    # capture (host work while the GPU waits) stays outside the timed region
    for _ in range(max(args.warmup, 3)):
        one_step()
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps (outside each step's event pair)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        one_step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = sum(step_ms) / len(step_ms)
    if pg:
        ms = aggregate_ms(pg, ms, dev)
        pg.barrier()
    value = ws * 1000.0 / ms

    # the other precision modes on the same input (device timing as above)
    def time_mode(prec, steps, interpolation="charge"):
        g = FMM(s["L"], True, s["p"], s["depth"], precision=prec, interpolation=interpolation)
        g.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
        Eg, Fg, dVg, _ = g.outputs(dev)
        for _ in range(3):
            g.eval_into(t["x"], Eg, Fg, dVg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tms = []
        for _ in range(steps):
            flush.zero_()
            e0.record(stream)
            g.eval_into(t["x"], Eg, Fg, dVg)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        m2l_alone = None
        if prec == "fp32":  # the CUDA-core M2L alone (every level), for its roofline
            g.set_profiling(True, serial=True)
            runs = []
            for _ in range(3):
                flush.zero_()
                g.eval_into(t["x"], Eg, Fg, dVg)
                runs.append(g.stage_times()["m2l"])
            g.set_profiling(False)
            m2l_alone = statistics.median(runs)
        g.close()
        return ws * 1000.0 / (sum(tms) / len(tms)), (Eg, Fg, dVg), m2l_alone

    modes = {precision: {"evals_per_s": value, "out": (E, F, dV)}}
    for prec in ("fp32", "tf32", "3xtf32", "3xbf16", "fp16"):
        if prec not in modes:
            try:
                v, o, m2l_alone = time_mode(prec, min(args.steps, 10))
                modes[prec] = {"evals_per_s": v, "out": o}
                if m2l_alone:
                    modes[prec]["m2l_alone_ms"] = m2l_alone
            except Exception as exc:  # mode not offered for this p / depth
                modes[prec] = {"error": str(exc)}
    # sites with two lambda coordinates over four charge forms (Sec. 2.1 Eq. 2): half the sites
    # get a tautomer; the same atoms and positions, in the default precision
    s4 = synth.tautomer_sites(s, seed=9, tautomer_fraction=0.5)
    tname = precision + "+tautomers"
    try:
        g4 = FMM(s["L"], True, s["p"], s["depth"], precision=precision)
        t4 = {k: torch.from_numpy(np.ascontiguousarray(s4[k])).to(dev) for k in ("qA", "qB", "qC", "qD", "lam")}
        g4.set_charges4(t4["qA"], t4["qB"], t4["qC"], t4["qD"], t["site"], t4["lam"])
        E4, F4, dV4, _ = g4.outputs(dev)
        for _ in range(3):
            g4.eval_into(t["x"], E4, F4, dV4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tms = []
        for _ in range(min(args.steps, 10)):
            flush.zero_()
            e0.record(stream)
            g4.eval_into(t["x"], E4, F4, dV4)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        g4.close()
        modes[tname] = {"evals_per_s": ws * 1000.0 / (sum(tms) / len(tms)), "out": (E4, F4, dV4), "system": s4}
    except Exception as exc:
        modes[tname] = {"error": str(exc)}
    # the Hamiltonian-interpolation form (intra-site correction, Sec. 2.1 Eq. 1) in the default precision
    hname = precision + "+hamiltonian"
    try:
        v, o, _ = time_mode(precision, min(args.steps, 10), interpolation="hamiltonian")
        modes[hname] = {"evals_per_s": v, "out": o, "hamiltonian": True}
    except Exception as exc:
        modes[hname] = {"error": str(exc)}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region:
    # every step copies its positions to the device and its E, F and dV/dlambda back.  The
    # headline uses fmm_eval_host_async with K calls in flight on two streams in turn, timed from
    # the first call to the synchronisation after the last: a call's position copy overlaps the
    # previous call's evaluation, and its result copies overlap the next call's evaluation (the
    # handle orders its evaluations across the two streams).  Before each call its stream waits
    # for the end of the previous evaluation's kernels (fmm_stream_wait_eval) and then flushes
    # L2, so the flush sits between consecutive evaluations.  e2e_1stream: the same calls on one
    # stream (the result copies then delay the next evaluation); e2e_sync: the synchronous
    # fmm_eval_host, one call at a time.
    e2e = None
    if not args.no_e2e:
        # page-locked host buffers from the library's allocator (see fmm_host_alloc)
        from paper_2410_01626_b300 import pinned_empty
        xh = pinned_empty((n, 3))
        xh.copy_(torch.from_numpy(np.ascontiguousarray(s["x"])))
        Eh = [pinned_empty(1, torch.float64) for _ in range(2)]
        Fh = [pinned_empty((n, 3)) for _ in range(2)]
        dVh = [pinned_empty(max(K, 1)) for _ in range(2)]
        for _ in range(3):
            f.eval_host(xh, Eh[0], Fh[0], dVh[0])
        e_ms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            f.eval_host(xh, Eh[0], Fh[0], dVh[0])
            e_ms.append((time.perf_counter() - a) * 1e3)
        em_sync = sum(e_ms) / len(e_ms)
        for _ in range(3):
            f.eval_host_async(xh, Eh[0], Fh[0], dVh[0])
        # the pipelined figures: the median of three runs of K calls each (a run is a few ms of
        # host-side enqueueing, which a stall of the host thread can stretch)
        reps = []
        for _ in range(3):
            torch.cuda.synchronize()
            a = time.perf_counter()
            for _ in range(args.steps):
                flush.zero_()  # on the same stream, between the calls (inside the timed region)
                f.eval_host_async(xh, Eh[0], Fh[0], dVh[0])
            torch.cuda.synchronize()
            reps.append((time.perf_counter() - a) * 1e3 / args.steps)
        em_one = statistics.median(reps)
        streams = (torch.cuda.Stream(), torch.cuda.Stream())

        def call2(k):
            with torch.cuda.stream(streams[k & 1]):
                f.stream_wait_eval()  # after the previous evaluation's kernels (its copies run beside)
                flush.zero_()         # L2 flushed between the two evaluations
                f.eval_host_async(xh, Eh[k & 1], Fh[k & 1], dVh[k & 1])

        for k in range(4):
            call2(k)
        reps = []
        for _ in range(3):
            torch.cuda.synchronize()
            a = time.perf_counter()
            for k in range(args.steps):
                call2(k)
            torch.cuda.synchronize()
            reps.append((time.perf_counter() - a) * 1e3 / args.steps)
        em = statistics.median(reps)
        em_runs = reps
        if pg:
            em = aggregate_ms(pg, em, dev)
            em_one = aggregate_ms(pg, em_one, dev)
            em_sync = aggregate_ms(pg, em_sync, dev)
        e2e = {"value": ws * 1000.0 / em, "unit": "evals/s", "h2d_bytes_per_step": 12 * n,
               "d2h_bytes_per_step": 8 + 12 * n + 4 * K, "ms_per_step": em,
               "api": f"fmm_eval_host_async, {args.steps} calls in flight on two streams in turn, then one "
                      "synchronisation; median of three such runs",
               "ms_per_step_runs": em_runs,
               "l2": "flushed between consecutive evaluations (a 256 MiB write, timed, after "
                     "fmm_stream_wait_eval on the next call's stream)",
               "e2e_1stream": {"value": ws * 1000.0 / em_one, "unit": "evals/s", "ms_per_step": em_one,
                               "api": "fmm_eval_host_async, calls in flight on one stream, L2 flushed between"},
               "e2e_sync": {"value": ws * 1000.0 / em_sync, "unit": "evals/s", "ms_per_step": em_sync,
                            "api": "fmm_eval_host (synchronises every call), L2 flushed before each"}}

    # roofline of the dominant kernel (M2L), live from the stage events
    peaks = load_peaks()
    nc = (s["p"] + 1) ** 2
    # the M2L launch the "m2l" stage times: every level, or with the tensor-core M2L the two
    # finest levels (the coarse levels then run on a side branch beside it)
    split = stages.get("m2l_coarse", 0.0) > 0.0
    lev = range(s["depth"] - 1, s["depth"] + 1) if split else range(1, s["depth"] + 1)
    boxes = sum(8 ** l for l in lev)
    m2l_flop = boxes * 189 * 2 * nc * nc
    m2l_ms = stages_alone.get("m2l", float("nan"))  # the kernel alone (L2 flushed before the step)
    achieved = m2l_flop / (m2l_ms * 1e-3) / 1e12
    sm_mhz = clocks.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1177.0)
    if precision == "fp32":
        # FP32 FMA pipe: 148 SMs x 128 lanes x 2 flop per clock, at the sampled SM clock
        peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"FP32 FMA: 148 SM x 128 lanes x 2 flop x {sm_mhz:.0f} MHz (sampled median)"}
    else:
        # the M2L launch is a sub-millisecond kernel, so the burst figure applies; the sustained
        # one (a seconds-long GEMM loop under the power cap) is reported beside it
        bf16 = peaks.get("bf16_tflops", 1738.8)
        bf16_sus = peaks.get("bf16_tflops_sustained", 1348.1)
        ratio = 1.0 if precision in ("3xbf16", "fp16") else 0.5  # 16-bit forms: the bf16 rate; TF32: half
        peak = bf16 * ratio
        src = ("measured burst bf16 cuBLAS, of measured" if ratio == 1.0 else
               "measured burst bf16 cuBLAS x 0.5 (nominal tf32/bf16 ratio), of measured")
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": src, "peak_sustained": bf16_sus * ratio,
                "frac_of_sustained": achieved / (bf16_sus * ratio)}
        # what the tensor pipe executes: 128 output rows x the K it multiplies -- ncp (padded
        # coefficients) once, three times in the split forms, and in the FP16 form once plus
        # one K step of 16 for the cross terms of the lowest coefficients
        ncp = 16 * ((nc + 15) // 16)
        keff = {"tf32": ncp, "3xtf32": 3 * ncp, "3xbf16": 3 * ncp, "fp16": ncp + 16}[precision]
        executed = boxes * 189 * 2.0 * 128 * keff
        roof["pipe_flop_per_launch"] = executed
        roof["pipe_frac"] = executed / (m2l_ms * 1e-3) / 1e12 / peak
    roof["traffic"] = m2l_traffic(precision)
    roof["kernel"] = "M2L, levels %d..%d" % (lev[0], lev[-1])
    roof["flop_per_launch"] = m2l_flop
    # the same interactions counted as a rotation-based O(p^3) M2L would do them (rotate,
    # translate along z, rotate back: about 6 (p + 1)^3 flop each), the minimal algorithmic
    # count, so that the dense formulation's extra work does not flatter the rate
    rot_flop = boxes * 189 * 6 * (s["p"] + 1) ** 3
    roof["flop_per_launch_rotation_count"] = rot_flop
    roof["achieved_rotation_count"] = rot_flop / (m2l_ms * 1e-3) / 1e12
    roof["ms_per_launch"] = m2l_ms
    roof["ms_in_step"] = stages.get("m2l")  # the same launch inside an ordinary step, sharing SMs

    # roofline of the near field (P2P), the kernel alone: 20 flop per ordered pair (3 sub, r^2
    # 3, q/r 1, potential 1, q/r^3 2, gradient 3 FMA = 13 FP32 operations, counted as the usual
    # 20 flop with the FMAs as two) against the FP32 pipe: 148 SMs x 128 lanes x 2 flop x clock
    counts = f.binning()[3].cpu().numpy().astype(np.int64)
    nb = 1 << s["depth"]
    grid = np.zeros((nb, nb, nb), np.int64)
    leaves = np.arange(len(counts))
    def compact(v):
        out = np.zeros_like(v)
        for b in range(s["depth"]):
            out |= ((v >> (3 * b)) & 1) << b
        return out
    grid[compact(leaves), compact(leaves >> 1), compact(leaves >> 2)] = counts
    nbsum = sum(np.roll(grid, (dx, dy, dz), (0, 1, 2)) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
    pairs = int((grid * nbsum).sum()) - n  # ordered pairs i != j over the 27 neighbour leaves
    p2p_ms = stages_alone.get("p2p", float("nan"))
    p2p_flop = 20.0 * pairs
    p2p_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    p2p_ach = p2p_flop / (p2p_ms * 1e-3) / 1e12
    roof_p2p = {"bound": "alu", "achieved": p2p_ach, "peak": p2p_peak, "unit": "TFLOP/s", "frac": p2p_ach / p2p_peak,
                "peak_source": f"FP32 FMA: 148 SM x 128 lanes x 2 flop x {sm_mhz:.0f} MHz (sampled median), derived",
                "kernel": "P2P near field (k_p2p), alone", "pairs": pairs, "flop_per_launch": p2p_flop,
                "ms_per_launch": p2p_ms, "ms_in_step": stages.get("p2p")}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(s, check_full=synth.solvated_30k() if not args.small else None)
        # accuracy of every mode against the FP64 oracle on sampled atoms (plus all site atoms,
        # so dV/dlambda is complete); E needs every atom and is compared between modes instead
        import oracle
        rng = np.random.default_rng(7)
        sample = rng.choice(n, 400, replace=False)
        a0 = time.perf_counter()
        ref = oracle.evaluate(s, targets=sample, tol=1e-8)
        cpu["accuracy_sample_seconds"] = time.perf_counter() - a0
        idx = ref["idx"]
        href = None
        if any(m.get("hamiltonian") for m in modes.values()):
            hc = oracle.hamiltonian_correction(s, tol=1e-8)  # plain pair sums over the sites
            href = {"F": ref["F"] + hc["F"][idx], "dVdl": ref["dVdl"] + hc["dVdl"]}
        for prec, m in modes.items():
            if "out" not in m:
                continue
            r = href if m.get("hamiltonian") else ref
            if "system" in m:  # four-form sites: their own oracle reference on the same atoms
                r = oracle.evaluate(m["system"], targets=sample, tol=1e-8)
            Em, Fm, dVm = m["out"]
            Fs = Fm.double().cpu().numpy()[idx]
            m["rel_err_vs_oracle"] = {
                "F_rms": float(np.sqrt(((Fs - r["F"]) ** 2).sum() / (r["F"] ** 2).sum())),
                "dVdl": float(np.linalg.norm(dVm.double().cpu().numpy() - r["dVdl"]) / np.linalg.norm(r["dVdl"])),
                "atoms_compared": int(len(idx))}
    m32 = modes.get("fp32", {})
    if m32.get("m2l_alone_ms"):  # the FP32 CUDA-core M2L (every level), alone, against the FP32 pipe
        f32_flop = sum(8 ** l for l in range(1, s["depth"] + 1)) * 189 * 2 * nc * nc
        f32_ach = f32_flop / (m32["m2l_alone_ms"] * 1e-3) / 1e12
        m32["roofline_m2l"] = {"bound": "alu", "achieved": f32_ach, "peak": p2p_peak, "unit": "TFLOP/s",
                               "frac": f32_ach / p2p_peak, "flop_per_launch": f32_flop,
                               "peak_source": roof_p2p["peak_source"],
                               "kernel": "FP32 CUDA-core M2L (k_m2l_f32 + k_sum8), every level, alone"}
    for prec, m in modes.items():
        if ("out" in m and prec != "fp32" and not m.get("hamiltonian") and "system" not in m
                and "out" in modes.get("fp32", {})):
            E32 = modes["fp32"]["out"][0].item()
            m["E_rel_diff_vs_fp32"] = abs(m["out"][0].item() - E32) / abs(E32)
        m.pop("out", None)
        m.pop("system", None)

    launches = f.launches_per_eval() * args.steps
    f.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "3xtf32": "tf32x3", "3xbf16": "bf16x3", "fp16": "f16"}[precision],
                "data": "synthetic",
                "config": {"workload": WORKLOAD if not args.small else "solvated_30k, p=10, depth 4",
                           "precision": precision, "atoms": n, "sites": K, "p": s["p"], "depth": s["depth"],
                           "l2": "flushed between steps (256 MiB write outside each step's event pair)",
                           "parallelism": f"replicas x{ws}"},
                "stages_ms": stages, "stages_alone_ms": stages_alone, "roofline": roof, "roofline_p2p": roof_p2p,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "wall_s_timed": wall1 - wall0,
                "step_ms_stats": step_stats(step_ms)}
        line["modes"] = modes
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def _timed_region(fn, steps, stream, local, flush=None):
    """Run fn() `steps` times between CUDA events (L2 flushed before each step when given);
    returns per-step ms and the sampled clocks."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    time.sleep(0.3)
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)], clk.stop()


def run_batch(args):
    """64 independent replicas (N log-uniform in 5k..50k) evaluated as one CUDA graph; depths
    chosen per replica by the autotuner."""
    import numpy as np
    import torch
    import synth
    from paper_2410_01626_b300 import Batch, FMM
    from paper_2410_01626_b300.autotune import TILES, tune
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = "fp16" if args.precision == "auto" else args.precision
    reps = synth.replicas(64, first_seed=100 + 64 * rank)
    solvers, xs, depths, cfgs = [], [], [], []
    for s in reps:
        t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in ("x", "qA", "qB", "site", "lam")}
        cfg, _ = tune(s["L"], True, s["p"], prec, t["x"], t["qA"], t["qB"], t["site"], t["lam"], reps=2, tiles=TILES)
        f = FMM(s["L"], True, s["p"], cfg["depth"], precision=prec, m2l_rows=cfg["m2l_rows"], p2p_warps=cfg["p2p_warps"])
        f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
        solvers.append(f)
        xs.append(t["x"])
        depths.append(cfg["depth"])
        cfgs.append(cfg)
    outs = [f.outputs(dev) for f in solvers]
    b = Batch(solvers)
    stream = torch.cuda.current_stream()
    fn = lambda: b.eval_into(xs, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    for _ in range(max(args.warmup, 3)):
        fn()
    ms_list, clocks = _timed_region(fn, args.steps, stream, local)
    ms = sum(ms_list) / len(ms_list)
    atoms = sum(len(s["x"]) for s in reps)
    line = {"metric": "replica FMM evals/s (64 replicas, 5k-50k atoms, one CUDA graph)", "value": ws * 64 * 1000.0 / ms,
            "unit": "replica-evals/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": "batch64: replicas seeds 100..163, periodic, p=8, autotuned depth and tiles "
                                   "(fastest within F and dV/dlambda error 0.7e-4 against an order-10 estimate)",
                       "atoms_total": atoms, "depths": depths, "tiles": [[c["m2l_rows"], c["p2p_warps"]] for c in cfgs],
                       "precision": prec,
                       "l2": "working set of all replicas (~0.6 GB) exceeds L2"},
            "atom_evals_per_s": ws * atoms * 1000.0 / ms,
            "gpu_launches": sum(f.launches_per_eval() for f in solvers) * args.steps, "clocks": clocks,
            "roofline": None, "cpu_baseline": None, "e2e": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    for f in solvers:
        f.close()
    return 0


def run_loop(args):
    """lambda dynamics on the 500k system: per step one FMM evaluation (CUDA graph) and one
    device Langevin step with the double-well / pH bias (Sec. 2.2-2.3; per-site pKa_ref drawn
    around the pH, barrier 5 kJ/mol, partition function correction); lambda is bound to the
    solver so charges refresh every step."""
    import numpy as np
    import torch
    import synth
    from paper_2410_01626_b300 import FMM, lambda_bias, lambda_step
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = "fp16" if args.precision == "auto" else args.precision
    s = synth.solvated_500k()
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in ("x", "qA", "qB", "site", "lam")}
    f = FMM(s["L"], True, s["p"], s["depth"], precision=prec)
    f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
    lam = t["lam"].clone()
    vel = torch.zeros_like(lam)
    pH = 5.0
    pka = np.random.default_rng(11).uniform(3.5, 6.5, len(s["lam"]))
    bias = lambda_bias(pH, pka, 5.0, device=dev)
    f.bind_lambda(lam)
    E, F, dV, _ = f.outputs(dev)
    f.eval_into(t["x"], E, F, dV)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            f.eval_into(t["x"], E, F, dV)
    torch.cuda.current_stream().wait_stream(cs)
    n_steps = 1000
    step = [0]

    def one():
        g.replay()
        lambda_step(lam, vel, dV, step[0], 5, first=(step[0] == 0), bias=bias)
        step[0] += 1

    for _ in range(max(args.warmup, 3)):
        one()
    torch.cuda.synchronize()
    a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    time.sleep(0.3)
    a.record()
    for _ in range(n_steps):
        one()
    b2.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = a.elapsed_time(b2) / n_steps
    lam_np = lam.cpu().numpy()
    line = {"metric": "lambda-dynamics steps/s (500k atoms: FMM eval + Langevin step, graph replay)",
            "value": ws * 1000.0 / ms, "unit": "steps/s", "n_gpus": ws, "steps": n_steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
            "data": "synthetic",
            "config": {"workload": "loop1000: " + WORKLOAD, "langevin": "BAOAB m=60 u, dt=2 fs, gamma=1/ps, 300 K",
                       "bias": "double well (barrier 5 kJ/mol) + pH 5 offset by partition function correction, "
                               "pKa_ref U(3.5, 6.5) per site",
                       "l2": "working set > L2 per step"},
            "lambda_range": [float(lam_np.min()), float(lam_np.max())],
            "deprotonated_fraction": float((lam_np > 0.5).mean()),
            "gpu_launches": (f.launches_per_eval() + 1) * n_steps, "clocks": clocks,
            "roofline": None, "cpu_baseline": None, "e2e": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    f.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "loop1000":
        return run_loop(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
