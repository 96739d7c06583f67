"""Benchmark of the ASCC / PLASCC solve on one GB300.

Default workload: one complete PLASCC solve with the mixed-triples slice T3'
(the paper's one-CSF ASCCSD, Sec. II.B.1, linearised as in Sec. II.C) of the
o=20, v=200 synthetic state (naux = 660, seed 0, excitation 19 -> 3, sigma
from the fixed coupling of synth/), from the zeroth-order guess to
max|R| <= 1e-8 and |dE| <= 1e-10 Eh, in mixed precision (split-BF16 tensor-core
contractions, FP64-class digit-plane polishing).  One step is one such solve;
`value` is solves per second (whole job: every replica's solves over the
slowest replica's time), measured with CUDA events on the context's stream
with the molecule's integrals already resident.  `e2e` is the same solve
requested through the host-buffer C ABI (context creation from pinned host
eps/B, integral setup, solve, energy back to the host).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload c1|c2|c3|batch|serve|gemm] [--precision mixed|fp64tc|fp64]
                    [--triples 0|1] [--fp64-solve]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("ASCC solves/sec & residual TFLOP/s vs plain FP64 at 1e-6 Eh; "
          "p50/p99 latency")
SERVE_NOTE = ("scaled-down serving trace: o log-uniform [5,20], v log-uniform [50,160], 1-4 "
              "excited states per molecule plus its ground state, Poisson arrivals")
WORKLOADS = {
    "c2": dict(o=20, v=200, seed=0, hole=19, particle=3),
    "c1": dict(o=4, v=20, seed=0, hole=3, particle=0),
    "c3": dict(o=30, v=300, seed=0, hole=29, particle=0),
}
FP64_NOMINAL_TFLOPS = 1.25


def workload_name(wl, triples):
    n = wl["o"] + wl["v"]
    return (f"ascc solve o={wl['o']} v={wl['v']} naux={3 * n} excitation "
            f"{wl['hole']}->{wl['particle']} (PLASCC{' + T3' + chr(39) if triples else ''}), "
            "max|R| <= 1e-8")


def measured_peaks():
    """Roofline denominators measured on this machine (MEASURED_PEAKS.json), else the
    fallback figures of the profiling recipe."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
                "bf16_sustained": float(d["bf16_tflops_sustained"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[5 + k].lower() in ("active", "1")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_residual_timer(wl, steps, warmup):
    """Seconds per oracle residual of the workload's state (list over the timed
    steps).  The sample is the oracle's T1/T2 residual (singles, doubles,
    partial linearisation, energy) at the zeroth-order guess: the oracle's
    evaluation of the T3' terms takes more than ten minutes per residual at
    o=20, v=200 on the host cores, far beyond a bounded sample, so the sample
    leaves them out and the derived solves/s is an upper bound for the oracle."""
    import synth
    from oracle import amplitudes as amp
    from oracle import ascc as oracle_ascc
    from oracle import spinadapted as sa
    o, v = wl["o"], wl["v"]
    s = synth.make_system(o, v, seed=wl["seed"])
    hbar, Bbar, _ = oracle_ascc.prepare(s.eps, s.B, o, wl["hole"], wl["particle"])
    t1, t2, _ = amp.initial_guess(o, v, wl["hole"], wl["particle"])
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        sa.residual(hbar, Bbar, o, t1, t2, linearize=True, hole=wl["hole"], particle=wl["particle"])
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
    return times


ORACLE_SAMPLE = ("one oracle T1/T2 residual of the same state at the zeroth-order guess per step "
                 "(the T3' terms left out: over ten minutes per residual on these cores), times the "
                 "iterations of a converged solve of that state -> an upper bound on the oracle's "
                 "solves/s")


def flops_per_residual(o, v, naux, excited=True, linearize=True):
    """Algorithmic flops of one residual of this path (2 per multiply-add).

    Counts the contractions the CUDA path performs (the same count the
    library accumulates in ascc_profile.gemm_flops), so the CPU baseline and
    the reference arm can be put on the same scale without a GPU.
    """
    n = o + v
    P = naux
    f = 0.0
    f += 2 * 2 * P * n ** 3 + 4 * n ** 3              # dressing L B R, L h R
    f += 2 * n * n * P + 2 * n * n * o * P             # J, K
    f += 2 * P * (o ** 4 + o ** 3 * v + 5 * o * o * v * v)  # DF blocks
    f += 2 * P * o * v * o * v + 2 * P * v * v * o      # singles DF term
    f += 2 * o ** 3 * v * v * 2                         # singles ooov, Fov
    f += 2 * o * o * v * v * n * v                      # dense ladder (xc|bd)
    nu = v + (1 if excited else 0)
    if excited:
        f += 3 * 2 * o * o * n * v * v                  # hole-slot corrections
    f += 2 * o * o * nu * nu * o * o                    # occupied ladder rows
    f += 2 * o * o * n * n * v + 2 * o * o * v * v * n  # L (x) L dressing
    f += 2 * o ** 4 * v * v                             # oooo x t
    f += 3 * 2 * o ** 3 * v ** 3                        # linear ring / crossed ring
    f += 2 * o * o * v ** 3 + 2 * o ** 3 * v * v        # linear Fock-like
    quad = 2 * o ** 4 * v * v * 2 + 2 * o ** 3 * v ** 3 * 5 + 2 * o ** 3 * v * v * 2 \
        + 2 * o * o * v ** 3 + 2 * o ** 3 * v * v
    f += quad * (2 if linearize else 1)
    f += 2 * o * o * v * v                              # energy
    return f


def oracle_iterations(name, default=50):
    path = os.path.join(ROOT, "tests", "golden", "reference_energies.txt")
    if os.path.exists(path):
        for line in open(path):
            if line.split() and line.split()[0] == name:
                return int(line.split()[8])
    return default


def run_reference(args, wl):
    """The CPU oracle as it stands, on the host cores: each step is one bounded
    sample (ORACLE_SAMPLE); ms_per_step is that sample's measured time, and the
    value converts it to solves/s with the iteration count of the solve."""
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    times = oracle_residual_timer(wl, args.steps, max(1, args.warmup))
    naux = 3 * (wl["o"] + wl["v"])
    name = f"{args.workload}_plascc_excited" + ("_t3" if args.triples else "")
    iters = oracle_iterations(name, default=SOLVE_ITERATIONS.get((args.workload, args.triples), 50))
    per = sum(times) / len(times)
    value = 1.0 / (per * iters)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * per, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(wl, args.triples), "o": wl["o"], "v": wl["v"],
                   "naux": naux, "excitation": [wl["hole"], wl["particle"]],
                   "method": "PLASCC" + ("+T3'" if args.triples else ""),
                   "sigma": _sigma(wl), "triples": int(args.triples),
                   "step": ORACLE_SAMPLE, "iterations_per_solve": iters},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": ORACLE_SAMPLE},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _sigma(wl):
    import synth
    return synth.default_sigma(wl["o"], wl["v"])


# iterations of the GPU solves of these states (FP64-class and mixed agree to
# a few), used when the oracle has no converged solve of the state
SOLVE_ITERATIONS = {("c2", 1): 63, ("c2", 0): 28}


# dram__bytes_read.sum + dram__bytes_write.sum of the pair-row ladder GEMM
# (3-product variant) per launch, from the last ncu capture at M=210 N=40000
# K=8192 (1.3246 GB + 0.1199 GB) scaled by 40000 / 8192; the kernel's store
# order changed after it, so the roofline reports traffic null and names
# this figure in its note
LADDER_TRAFFIC = {("c2", "mixed"): 7.05e9}

DTYPES = {"fp64": "f64", "mixed": "bf16x3-split/f64",
          "fp64tc": "f64 via bf16 digit-plane tensor-core products"}


def precision_code(pkg, name):
    return {"fp64": pkg.ASCC_FP64, "mixed": pkg.ASCC_MIXED_BF16, "fp64tc": pkg.ASCC_FP64_TC}[name]


def max_over_ranks(ms, dist=None, device="cpu"):
    """The timed region of a step is the slowest rank's (replicas share no data)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def golden_energy(name):
    path = os.path.join(ROOT, "tests", "golden", "reference_energies.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.split() and line.split()[0] == name:
            return float(line.split()[7])
    return None


def run_server_workload(args, kind):
    """Batched (64 molecules) or streamed (Poisson arrivals) solves through ascc_server."""
    import torch
    import synth
    import paper_2501_10515_gb300 as pkg
    torch.cuda.set_device(0)
    prec = precision_code(pkg, args.precision)
    if kind == "batch":
        reqs = []
        for w in synth.batch_workload(args.requests or 64):
            reqs.append(dict(o=w["o"], v=w["v"], seed=w["seed"], arrival=0.0,
                             states=[None] + list(w["excitations"])))
    else:
        trace = synth.serving_trace(args.requests or 40, seed=12345, rate=args.rate,
                                    o_range=(5, 20), v_range=(50, 160))
        reqs = [dict(o=r["o"], v=r["v"], seed=r["seed"], arrival=r["arrival"],
                     states=[None] + [(r["o"] - 1 - k % 2, k // 2) for k in range(len(r["excitations"]))])
                for r in trace]
    srv = pkg.Server(int(args.budget_gb * (1 << 30)), max_active=args.workers, precision=prec)
    t0 = time.perf_counter()
    sub = {}
    for q, r in enumerate(reqs):
        if kind == "serve":
            dt = r["arrival"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        s = synth.make_system(r["o"], r["v"], seed=r["seed"])
        rid = srv.submit(r["o"], r["v"], s.naux, s.eps, s.B, r["states"])
        sub[rid] = q
    srv.drain()
    wall = time.perf_counter() - t0
    res = srv.results()
    srv.close()
    per_req = {}
    for x in res:
        a = per_req.setdefault(x["request_id"], [x["t_arrival"], x["t_end"], 0, 0])
        a[1] = max(a[1], x["t_end"])
        a[2] += 1
        a[3] += int(x["status"] == 0)
    lat = np.array([b - a for a, b, _, _ in per_req.values()])
    failures = []
    for x in res:
        if x["status"] != 0 and len(failures) < 24:
            r = reqs[sub[x["request_id"]]]
            st = r["states"][x["state_index"]] if x["state_index"] >= 0 else "request"
            failures.append({"o": r["o"], "v": r["v"], "seed": r["seed"], "state": st,
                             "status": int(x["status"]), "iterations": int(x["iterations"])})
    solves = sum(v[2] for v in per_req.values())
    ok = sum(v[3] for v in per_req.values())
    line = {
        "metric": METRIC, "value": ok / wall, "unit": "solves/s", "n_gpus": 1,
        "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 * wall / max(1, len(reqs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": ("batched launch of 64 independent molecules, o in [4,16], v in "
                                "[40,160], 1-3 excitations each plus the ground state"
                                if kind == "batch" else SERVE_NOTE),
                   "workers": args.workers, "memory_budget_gb": args.budget_gb,
                   "arrival_rate_per_s": args.rate if kind == "serve" else None},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "requests": len(reqs), "states": solves, "converged_states": ok, "wall_s": wall,
        "not_converged": failures,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gemm(args):
    """One tensor-core GEMM alone, by default on the ladder's shape class (M = o^2 = 400,
    N = (o+v) v = 44000) with K = 4096, inputs larger than L2.  --level 1..3: split-BF16
    products; --level 4: FP64-class digit-plane products."""
    import torch
    import paper_2501_10515_gb300 as pkg
    M, N, K = (int(x) for x in args.gemm_shape.split(","))
    lev = args.level
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(M, K, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g)
    C = torch.zeros(M, N, device="cuda", dtype=torch.float64)
    call = ((lambda: pkg.gemm_fp64_tc(A, B, C)) if lev == 4 else
            (lambda: pkg.gemm_split_bf16(A, B, C, lev)))
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    products = {1: 1, 2: 3, 3: 6, 4: 21}[lev]
    tf = 2.0 * M * N * K / (ms / 1e3) / 1e12
    print(json.dumps({"kernel": ("digit-plane tcgen05 GEMM" if lev == 4 else "split-BF16 tcgen05 GEMM")
                      + " incl. operand split and K reduction",
                      "M": M, "N": N, "K": K, "level": lev, "products": products, "ms": ms,
                      "tflops_fp64_equivalent": tf, "mma_tflops": tf * products,
                      "mma_frac_of_bf16_burst": tf * products / measured_peaks()["bf16"],
                      "peak_source": measured_peaks()["source"]}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS) + ["batch", "serve", "gemm"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "fp64tc"])
    ap.add_argument("--triples", type=int, default=1, choices=[0, 1])
    ap.add_argument("--step", default="solve", choices=["solve", "iteration"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--fp64-iterations", type=int, default=2)
    ap.add_argument("--fp64-solve", action="store_true",
                    help="time one complete plain-FP64 solve of the same state (minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=0)
    ap.add_argument("--rate", type=float, default=1.0)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=180.0)
    ap.add_argument("--level", type=int, default=2)
    ap.add_argument("--diis", type=int, default=0,
                    help="DIIS history length (0: 32 with T3', whose amplitudes converge more "
                         "slowly, else the library default 16)")
    ap.add_argument("--gemm-shape", default="400,44000,4096")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload in ("batch", "serve"):
        return run_server_workload(args, args.workload)
    if args.workload == "gemm":
        return run_gemm(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import synth
    import paper_2501_10515_gb300 as pkg

    o, v = wl["o"], wl["v"]
    s = synth.make_system(o, v, seed=wl["seed"])
    stream = torch.cuda.current_stream()
    mixed = args.precision != "fp64"  # tensor-core contractions
    prec = precision_code(pkg, args.precision)
    diis = args.diis or (32 if args.triples else 16)
    ctx = pkg.Context(o, v, s.naux, s.eps, s.B, hole=wl["hole"], particle=wl["particle"],
                      linearize=1, triples=args.triples, stream=stream.cuda_stream, precision=prec,
                      diis_dim=diis)

    def one_unit():
        if args.step == "solve":
            ctx.reset()
            return ctx.iterate(ctx.options.max_iter + 1)
        return ctx.iterate(1)

    if args.step == "iteration":
        ctx.reset()
    for _ in range(args.warmup):
        one_unit()
    torch.cuda.synchronize()
    # kernel launches so far (this process has launched no others): lets an ncu
    # launch list skip to the timed region (-s)
    print(f"launches before the timed region: {ctx.launches()}", file=sys.stderr, flush=True)
    ctx.set_profiling(True)
    p0 = ctx.profile()
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    results = []
    evs[0].record(stream)
    for k in range(args.steps):
        results.append(one_unit())
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ctx.set_profiling(False)
    p1 = ctx.profile()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    ms = max_over_ranks(sum(per), dist, "cuda")
    units = world * args.steps
    flops = p1.gemm_flops - p0.gemm_flops
    tflops = world * flops / (ms / 1e3) / 1e12
    nlad = max(1, p1.ladder_launches - p0.ladder_launches)
    lad_ms = (p1.ladder_ms - p0.ladder_ms) / nlad
    lad_fl = (p1.ladder_flops - p0.ladder_flops) / nlad
    lad_mma = (p1.ladder_mma_flops - p0.ladder_mma_flops) / nlad
    achieved = lad_fl / (lad_ms / 1e3) / 1e12
    mma_rate = lad_mma / (lad_ms / 1e3) / 1e12
    peaks = measured_peaks()
    if mixed:
        # the ladder launch is timed inside a seconds-long solve: the sustained figure
        peak, bound = peaks["bf16_sustained"], "tensor"
        peak_note = (f"BF16 dense, sustained under the power cap, of {peaks['source']} "
                     "(MEASURED_PEAKS.json bf16_tflops_sustained)")
    else:
        peak, bound = FP64_NOMINAL_TFLOPS, "alu"
        peak_note = "nominal FP64 rate of the recipe table (no FP64 peak is measured on this pool)"
    last = results[-1]
    iters = last.iterations
    value = units / (ms / 1e3) if args.step == "solve" else tflops
    unit = "solves/s" if args.step == "solve" else "TFLOP/s"
    gname = f"{args.workload}_plascc_excited" + ("_t3" if args.triples else "")
    ref_e = golden_energy(gname)

    # the plain FP64 path on the same state (a sibling context sharing the
    # molecule): a few iterations always, the complete solve with --fp64-solve
    fp64 = None
    if mixed and args.step == "solve" and (args.fp64_iterations > 0 or args.fp64_solve):
        cf = pkg.Context(o, v, s.naux, None, None, hole=wl["hole"], particle=wl["particle"],
                         base=ctx, linearize=1, triples=args.triples, stream=stream.cuda_stream,
                         precision=pkg.ASCC_FP64, diis_dim=diis)
        cf.reset()
        cf.iterate(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        nit = max(1, args.fp64_iterations)
        e0.record(stream)
        cf.iterate(nit)
        e1.record(stream)
        torch.cuda.synchronize()
        fms = e0.elapsed_time(e1) / nit
        fp64 = {"ms_per_iteration": fms, "iterations_timed": nit}
        if args.fp64_solve:
            torch.cuda.synchronize()
            e0.record(stream)
            rf = cf.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            fp64.update(solve_s=e0.elapsed_time(e1) / 1e3, solve_iterations=rf.iterations,
                        solve_status=int(rf.status), solve_energy=rf.energy,
                        solves_per_s=1e3 / e0.elapsed_time(e1),
                        energy_difference_to_this_solve=abs(rf.energy - last.energy))
        else:
            fp64.update(solve_s_estimate=fms * iters / 1e3,
                        note="estimate: FP64 time per iteration measured on this state x this "
                             "solve's iterations; python bench.py --fp64-solve times the whole solve")
        cf.close()

    # the timed context is released before the end-to-end request, which
    # builds its own molecule (two copies of the large ladder blocks need not fit)
    ctx.close()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    eps_p, B_p = pin(s.eps), pin(s.B)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_energy = None
    for _ in range(args.e2e_steps):
        c2 = pkg.Context(o, v, s.naux, eps_p, B_p, hole=wl["hole"], particle=wl["particle"],
                         linearize=1, triples=args.triples, precision=prec, diis_dim=diis)
        r2 = c2.solve()
        e2e_energy = r2.energy
        c2.close()
    e2e_s = (time.perf_counter() - t0) / max(1, args.e2e_steps)

    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": workload_name(wl, args.triples), "o": o, "v": v, "naux": s.naux,
                   "excitation": [wl["hole"], wl["particle"]],
                   "method": "PLASCC" + ("+T3'" if args.triples else ""),
                   "triples": int(args.triples), "sigma": s.sigma,
                   "n_t3": int(n3_of(wl, args.triples)),
                   "precision": args.precision, "diis_dim": diis, "parallelism": f"replicas{world}",
                   "l2": ("inputs larger than L2: the (xc|bd) block (%.1f GB as 3 BF16 planes, "
                          "%.1f GB as 6 digit planes, %.1f GB FP64) is streamed every iteration"
                          % (6.0 * (o + v) * v ** 3 / 1e9, 12.0 * (o + v) * v ** 3 / 1e9,
                             8.0 * (o + v) * v ** 3 / 1e9)),
                   "step": ("one complete solve from the zeroth-order guess to max|R| <= 1e-8, "
                            "|dE| <= 1e-10" if args.step == "solve" else
                            "one solve iteration (residual + convergence test + Jacobi + DIIS)")},
        "clocks": clocks,
        "e2e": {"value": (1.0 / e2e_s) if (args.step == "solve" and args.e2e_steps) else None,
                "unit": "solves/s",
                "h2d_bytes_per_step": int(eps_p.nbytes + B_p.nbytes), "d2h_bytes_per_step": 56},
        "gpu_launches": int(p1.launches - p0.launches),
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "traffic_note": ("null: the epilogue's store order changed after the last "
                                      "ncu capture (the same bytes by construction, not "
                                      "captured again); that capture (profiles/, K = 8192, "
                                      "scaled to K = v^2) gave %.3g bytes per 3-product launch"
                                      % LADDER_TRAFFIC[(args.workload, args.precision)]
                                      if (args.workload, args.precision) in LADDER_TRAFFIC
                                      else None),
                     "kernel": {"fp64": "gemm_f64_kernel", "mixed": "gemm_tc_kernel",
                                "fp64tc": "gemm_oz_kernel"}[args.precision] +
                               " (the particle-particle ladder's pair-row GEMM, M = o(o+1)/2, "
                               "N = K = v^2, with its split-K reduction: the largest single launch)",
                     "peak_source": peak_note,
                     "achieved_note": "algorithmic flops of that launch, 2 o(o+1)/2 v^4 (one "
                                      "product per multiply-add), over its CUDA-event time on "
                                      "the state's stream, averaged over the launches of the "
                                      "timed solves; mma_* count every BF16 plane product",
                     "mma_tflops": mma_rate,
                     "mma_frac": mma_rate / peak,
                     "ladder_ms_share_of_step": (p1.ladder_ms - p0.ladder_ms) / (ms / world)},
        "residual_tflops": tflops,
        "residual_frac": tflops / world / peak,
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                       "note": "per solve, back to back on one state (not a serving latency: "
                               "see --workload serve)"},
        "iterations": iters, "iterations_low_precision": last.iterations_low,
        "status": int(last.status), "energy": last.energy,
        "energy_error_vs_oracle": (abs(last.energy - ref_e) if ref_e is not None else None),
        "oracle_energy_source": (f"tests/golden/reference_energies.txt {gname}"
                                 if ref_e is not None else
                                 ("none: the oracle's solve with T3' at this size is not "
                                  "feasible on the host; tests/test_gpu_fullsize.py checks this "
                                  "residual against tests/golden/c2_t3_residual.txt instead"
                                  if args.triples else
                                  "none: no oracle solve of this state is stored (the host has no "
                                  "room for its FP64 (vv|vv) block); tests/test_gpu_c3_mixed.py "
                                  "holds the mixed energy to the FP64-class one")),
        "e2e_energy": e2e_energy,
        "fp64_path": fp64,
    }
    if rank == 0 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        times = oracle_residual_timer(wl, 1, 0)
        ores = times[0]
        cb = {"cores": cores, "kind": "oracle", "sample": ORACLE_SAMPLE,
              "seconds_per_sample": ores, "iterations": iters}
        if args.step == "solve":
            cb.update(value=1.0 / (ores * iters), unit="solves/s")
        else:
            cb.update(value=flops_per_residual(o, v, s.naux) / ores / 1e12, unit="TFLOP/s")
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def n3_of(wl, triples):
    if not triples:
        return 0
    o, v = wl["o"], wl["v"]
    return (o - 1) * (v * (v - 1) // 2 + (v - 1) ** 2) + (o - 1) * (o - 2) // 2 * (v - 1) + \
        (o - 1) ** 2 * (v - 1)


if __name__ == "__main__":
    sys.exit(main())
