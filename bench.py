"""Benchmark of the parallel pulling protocol hot path on GB300.

One step = the whole PPP workload of the 104-bead chain: 21 windows x 32
replicas, 4e5 BAOAB steps each (0.4 ns at 1 fs), x recorded every 100 steps,
then the FP64 reductions into dF_JE / dF_fluct / dF_G / dF_com.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is replica-steps/s of the whole job
with inputs resident on the device; `e2e` is the same metric through the C
ABI with host buffers (system upload, run, result download inside the timed
region); `roofline` reports the chain kernel against the FP32 ALU peak;
`cpu_baseline` times the FP64 oracle on a bounded sample on the host cores.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "chain104_ppp"
N_BEADS = 104


def flops_per_replica_step(n: int) -> int:
    """Algorithmic FP32 flops of one BAOAB step of an n-bead chain (FMA = 2):
    36 per nonbonded pair (|i-j| >= 3), 20 per bond, 60 per angle, 110 per
    three-term dihedral, 33 per bead for the B, A, O, A, B updates."""
    pairs = n * (n - 1) // 2 - (2 * n - 3)
    return 36 * pairs + 20 * (n - 1) + 60 * (n - 2) + 110 * (n - 3) + 33 * n


def workload_config(run, world=1):
    """The `config` of the default line, shared by both arms."""
    return {"workload": WORKLOAD, "beads": N_BEADS, "windows": int(run.lambdas.size),
            "replicas_per_window": run.replicas, "md_steps_per_window": run.n_steps, "dt_ps": run.dt,
            "sample_stride": run.stride, "forces": "fp32", "reductions": "fp64",
            "parallelism": f"replicas x{world}", "l2": "256 MB flush between timed steps"}


def _workload(n_steps=None):
    from paper_1105_4840_gb300 import inputs

    w = inputs.chain_workload()
    if n_steps is not None:
        w["run"].n_steps = n_steps
        w["run"].n_equil = n_steps // 10
    return w


class ClockSampler:
    """nvidia-smi SM clock / throttle samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _ncu_traffic(warps):
    """DRAM bytes per chain-kernel launch from the committed ncu summary, only
    if it was taken on the current kernel source and the same warp count."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "chain_kernel_traffic.json")) as fh:
            t = json.load(fh)
        with open(os.path.join(ROOT, "paper_1105_4840_gb300", "csrc", "chain.cu"), "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    if t.get("chain_cu_sha256") != h or f"<float, {warps}>" not in t.get("kernel", ""):
        return None
    return t


def samples_per_replica(run):
    """x samples each replica records: every `stride` steps after `n_equil`."""
    return (run.n_steps - run.n_equil) // run.stride


def _reduction_roofline(ms, n_samples, peaks, fp64_tflops):
    """The reductions of one step against HBM (4 bytes of x per sample, read
    by each of stage 1's two passes) and beside the measured FP64 rate:
    stage 1 forms its exponentials and per-thread sums in double-float
    arithmetic on the FP32 pipe; three dependent launches of a few tens of
    microseconds, not HBM, bound the whole."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = 4.0 * n_samples / (ms * 1e-3) / 1e9
    return {"kernels": "partial_kernel, window_kernel, profile_kernel", "ms": ms, "samples": n_samples,
            "bound": "latency", "achieved_gbs": gbs, "hbm_peak_gbs": hbm, "hbm_frac": gbs / hbm,
            "ns_per_sample": ms * 1e6 / n_samples, "fp64_tflops_measured": fp64_tflops,
            "note": "stage 1 in double-float arithmetic on the FP32 pipe (FP64 per flush of 16 samples and in the "
                    "block trees); three dependent launches, not HBM, bound the reduction"}


def cpu_baseline(budget_s=12.0, n_steps=200, single_thread=True):
    """The FP64 oracle as it stands, on the host cores: replicas of the
    104-bead chain (windows round-robin), one thread per core; with
    single_thread, also the same oracle on one thread for the per-core
    figure."""
    import concurrent.futures as cf

    from oracle import _clib

    w = _workload()
    p, start, run = w["params"], w["start"], w["run"]
    ch = _clib.Chain(p)
    cores = os.cpu_count() or 1
    lam = run.lambdas

    def one(uid):
        ch.run(start, lam[uid % lam.size], run.k, run.kT, run.dt, run.gamma, n_steps, n_steps, 1,
               run.seed, uid)
        return n_steps

    done = 0
    t0 = time.perf_counter()
    uid = 0
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        while time.perf_counter() - t0 < budget_s:
            futs = [ex.submit(one, uid + i) for i in range(cores)]
            uid += cores
            done += sum(f.result() for f in futs)
    el = time.perf_counter() - t0
    out = {"value": done / el, "unit": "replica-steps/s", "cores": cores, "kind": "oracle",
           "sample": f"{uid} replicas x {n_steps} BAOAB steps of the 104-bead chain (FP64, "
                     f"{cores} threads, {el:.1f} s)",
           "replica_steps": done, "seconds": el}
    if not single_thread:
        return out
    done1, n1 = 0, 0
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < min(2.0, budget_s / 4):
        done1 += one(uid + n1)
        n1 += 1
    el1 = time.perf_counter() - t1
    out["single_thread"] = {"value": done1 / el1, "sample": f"{n1} replicas x {n_steps} steps on one thread"}
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    # every step is a bounded sample of the workload (about 6 s of oracle
    # work on all host cores); ms_per_step is the measured time of one such
    # step and value the replica-steps of all timed steps over their time
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(budget_s=1.0, single_thread=False)
    t0 = time.perf_counter()
    for q in range(args.steps):
        vals.append(cpu_baseline(budget_s=6.0, single_thread=(q == args.steps - 1)))
    el = time.perf_counter() - t0
    work = sum(b["replica_steps"] for b in vals)
    v = work / sum(b["seconds"] for b in vals)
    line = {"impl": "reference", "metric": "replica-steps/s", "value": v, "unit": "replica-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / max(args.steps, 1), "extrapolated": False,
            "step_work": f"a bounded sample of {work // max(args.steps, 1)} replica-steps per step "
                         "(the whole workload is 21 x 32 x 4e5 = 2.69e9 replica-steps)",
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(_workload().get("run"), world),
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "replica-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _nvtx(torch, name):
    """Open (name) or close (None) an NVTX range around a timed region, so
    that a profiler can select exactly its launches; a torch build without
    NVTX markers skips them."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except (RuntimeError, AttributeError):
        pass


def bench_batch(args, pmf, torch, stream):
    """Many uneven paths at once: 64 chains (40-400 beads), 21-61 windows
    each, 16 replicas, in the launch the batch autotuner picks (by default
    one packed persistent launch per chunk for the whole batch, else a CUDA
    graph of per-chain launches), then the per-chain FP64 reductions.
    Single GPU, rank 0 only."""
    from paper_1105_4840_gb300 import inputs

    bw = inputs.batch_workload(n_steps=args.md_steps)
    run, params, lams = bw["run"], bw["params"], bw["lambdas"]
    sysh = pmf.pmf_create_system_chain(params, bw["starts"])
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    tune_ms = rr.batch_autotune(min(run.n_steps, 1000))  # untimed setup
    binfo = rr.batch_launch()
    R = run.replicas
    replica_steps = sum(l.size for l in lams) * R * run.n_steps
    flops = sum(flops_per_replica_step(p.n) * l.size * R * run.n_steps for p, l in zip(params, lams))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def reduce_all():
        for m, l in enumerate(lams):
            rr.free_energy_item(m, l.size)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        rr.launch()
        rr.wait()
    reduce_all()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.5)
    sim_ms, red_ms = [], []
    _nvtx(torch, "timed")
    for i in range(args.steps):
        flush.fill_(float(i))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(stream)
        rr.launch()
        e[1].record(stream)
        rr.wait()
        reduce_all()  # synchronous per item: the host loop waits on each copy-out
        e[2].record(stream)
        torch.cuda.synchronize()
        sim_ms.append(e[0].elapsed_time(e[1]))
        red_ms.append(e[1].elapsed_time(e[2]))
    _nvtx(torch, None)
    clocks.stop()
    rr.wait()
    t_step = statistics.mean(a + b for a, b in zip(sim_ms, red_ms))
    clk = clocks.summary()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    peak = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    sim = statistics.mean(sim_ms)
    achieved = flops / (sim / 1000.0) / 1e12
    packed = binfo["mode"] == pmf.PMF_BATCH_PACKED
    chunks = math.ceil(run.n_steps / 100000) if packed else sum(math.ceil(run.n_steps / 100000) for _ in lams)
    n = [p.n for p in params]
    teams = {int(g): int(np.sum(binfo["teams"] == g)) for g in sorted(set(binfo["teams"].tolist()))}
    line = {"metric": "replica-steps/s", "value": replica_steps / (t_step / 1000.0), "unit": "replica-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch64_uneven", "chains": len(params), "beads_min": min(n),
                       "beads_max": max(n), "beads_total": sum(n), "windows_total": sum(l.size for l in lams),
                       "replicas_per_window": R, "md_steps_per_window": run.n_steps,
                       "launch": ("one packed persistent launch per 1e5-step chunk: %d CTAs of 16 warps, %d packs, "
                                  "policy %d, chains per team size %s" % (binfo["ctas"], binfo["packs"],
                                                                          binfo["policy"], teams))
                       if packed else "one CUDA graph, one branch per chain",
                       "autotune_probe_ms": tune_ms, "l2": "256 MB flush between timed steps"},
            "gpu_launches": args.steps * (chunks + 3 * len(lams)),
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons")},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "chain_pack_kernel<float>" if packed else "chain_kernel<float,4> (64 launches)",
                         "launch_ms": sim},
            "simulation_ms": sim, "reduction_ms": statistics.mean(red_ms)}
    print(json.dumps(line), flush=True)


def bench_precision(args, pmf, torch):
    """FP32 vs FP64 integration on the 104-bead workload with many replicas
    (same seeds, same uids): per window pair, the JE increments of both runs
    and their difference in units of the combined jackknife standard error;
    the same for the full path; the wall time of each run."""
    w = _workload(args.md_steps)
    p, start, run = w["params"], w["start"], w["run"]
    run.replicas = args.replicas
    lam = run.lambdas
    out = {}
    for prec, name in ((0, "fp32"), (1, "fp64")):
        sysh = pmf.pmf_create_system_chain([p], [start], precision=prec)
        rr = pmf.pmf_run_prepare(sysh, lam, pmf.make_params(run))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr.launch()
        rr.wait()
        el = time.perf_counter() - t0
        out[name] = {"res": rr.free_energy(), "seconds": el}
        rr.close()
        sysh.close()

    def incr(res):
        return np.diff(res["dF_JE"]), np.sqrt(np.maximum(np.diff(res["se_JE"] ** 2), 0.0))

    j32, s32 = incr(out["fp32"]["res"])
    j64, s64 = incr(out["fp64"]["res"])
    z = (j32 - j64) / np.hypot(s32, s64)
    kT = run.kT
    e32 = (float(out["fp32"]["res"]["dF_JE"][-1]), float(out["fp32"]["res"]["se_JE"][-1]))
    e64 = (float(out["fp64"]["res"]["dF_JE"][-1]), float(out["fp64"]["res"]["se_JE"][-1]))
    line = {"workload": "chain104_precision", "replicas_per_window": run.replicas, "windows": int(lam.size),
            "md_steps_per_window": run.n_steps, "kT": kT,
            "fp32_seconds": out["fp32"]["seconds"], "fp64_seconds": out["fp64"]["seconds"],
            "path_dF_JE": {"fp32": e32, "fp64": e64},
            "path_diff_kT": (e32[0] - e64[0]) / kT,
            "path_z": (e32[0] - e64[0]) / math.hypot(e32[1], e64[1]),
            "max_abs_z": float(np.max(np.abs(z))), "max_abs_diff_kT": float(np.max(np.abs(j32 - j64)) / kT),
            "per_window_pair": [{"pair": [float(lam[i]), float(lam[i + 1])], "dJE_fp32": float(j32[i]),
                                 "dJE_fp64": float(j64[i]), "se_fp32": float(s32[i]), "se_fp64": float(s64[i]),
                                 "z": float(z[i])} for i in range(lam.size - 1)]}
    print(json.dumps(line), flush=True)


def ladder_summary(rs, seeds, F_ref, kT, tolerances=(0.2, 0.3, 0.5, 1.0)):
    """GPU-seconds to a path free energy within eps of the reference: per
    seed, the run at the shortest tau from which this and every longer run
    stays within eps * kT of F_ref (None if none does); the median over the
    seeds only when every seed got there.  Also the mean deviation, its
    spread over the seeds, the mean jackknife SE and the mean GPU-seconds
    per tau.  rs: rows {"seed", "tau_ps", "gpu_s", "dF", "se"}."""
    def reach(eps):
        per_seed = []
        for seed in seeds:
            ladder = sorted([r for r in rs if r["seed"] == seed], key=lambda r: r["tau_ps"])
            ok = [abs(r["dF"] - F_ref) < eps * kT for r in ladder]
            first = next((i for i in range(len(ladder)) if all(ok[i:])), None)
            per_seed.append(None if first is None else {"tau_ps": ladder[first]["tau_ps"],
                                                        "gpu_s": ladder[first]["gpu_s"]})
        got = [x["gpu_s"] for x in per_seed if x is not None]
        return per_seed, (statistics.median(got) if got and len(got) == len(per_seed) else None), len(got)

    per_seed, med, n_ok = reach(0.2)
    by_tau = []
    for tau in sorted({r["tau_ps"] for r in rs}):
        d = np.array([(r["dF"] - F_ref) / kT for r in rs if r["tau_ps"] == tau])
        g = [r["gpu_s"] for r in rs if r["tau_ps"] == tau]
        se = [r["se"] / kT for r in rs if r["tau_ps"] == tau]
        by_tau.append({"tau_ps": tau, "bias_kT": float(d.mean()), "sd_kT": float(d.std(ddof=1)) if d.size > 1 else 0.0,
                       "mean_se_kT": float(np.mean(se)), "gpu_s": float(np.mean(g))})
    by_eps = []
    for eps in tolerances:
        ps, m, k = reach(eps)
        by_eps.append({"eps_kT": eps, "median_gpu_s": m, "seeds_within": k, "per_seed": ps})
    return {"median_gpu_s": med, "seeds_converged": n_ok, "per_seed": per_seed, "by_tau": by_tau, "by_eps": by_eps}


def bench_adaptive(args, pmf, torch):
    """GPU-seconds to a path free energy within 0.2 kT of a converged
    reference: the learned window placement (11 windows, surrogate-guided
    insertion with seeding; with continuation every round runs all windows in
    one launch, the current ones resuming from their replicas' end states)
    against the uniform 21-window grid, over a ladder of window relaxation
    times and several dynamics seeds.  The reference continues a dense
    uniform grid for a fixed number of rounds (each round resumes every
    replica from its end state with fresh noise) and averages its last
    rounds; their drift per round is reported beside it."""
    from paper_1105_4840_gb300 import inputs

    out = {"workload": "chain_adaptive_vs_uniform", "criterion_kT": 0.2, "chains": []}
    for n_beads in args.adaptive_beads:
        aw = inputs.adaptive_workload(n_beads)
        if args.tau_ps:
            aw["tau_ps"] = list(args.tau_ps)
        if args.tau_uniform_extra is not None:
            aw["tau_uniform_extra"] = list(args.tau_uniform_extra)
        if args.seeds:
            aw["seeds"] = list(args.seeds)
        p, start, run = aw["params"], aw["start"], aw["run"]
        R = args.adaptive_replicas or run.replicas
        kT = run.kT
        sysh = pmf.pmf_create_system_chain([p], [start])

        def steps_of(tau_ps):
            return int(round(tau_ps / run.dt))

        def timed(fn):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record()
            res = fn()
            ev[1].record()
            torch.cuda.synchronize()
            return res, ev[0].elapsed_time(ev[1]) / 1000.0

        def uniform(s, reps, n_steps, seed, uid_base=0, starts=None):
            lam = np.linspace(aw["lo"], aw["hi"], s)
            run.replicas, run.n_steps, run.n_equil, run.seed = reps, n_steps, n_steps // 10, seed
            pr = pmf.make_params(run, uid_base=uid_base)
            if starts is None:
                rr = pmf.pmf_run_prepare(sysh, lam, pr)
            else:
                rr = pmf.pmf_run_prepare_seeded(sysh, lam, pr, starts)

            def go():
                rr.launch()
                rr.reduce()
                rr.wait()
                return rr.free_energy()

            res, gs = timed(go)
            return res, gs, rr

        # converged reference: a dense uniform grid continued round after
        # round from its own end states; the mean of its last rounds, with
        # the least-squares drift per round over those rounds
        s_ref = aw["s_reference_cont"]
        r_ref = args.reference_replicas or aw["replicas_reference"]
        n_rounds = aw["reference_rounds"] if args.reference_rounds is None else args.reference_rounds
        n_avg = min(args.reference_average or aw["reference_average"], n_rounds)
        tau_ref = steps_of(aw["reference_round_ps"]) if args.reference_steps is None else args.reference_steps
        drift, ref_gpu_s, rr = [], 0.0, None
        if n_rounds == 0:  # no reference (the protocols' values alone)
            n_avg = 0
        for rnd in range(n_rounds):
            pos = None
            if rr is not None:
                pos, _ = rr.final_state()
                rr.close()
            res, gs, rr = uniform(s_ref, r_ref, tau_ref, 1000 + rnd, uid_base=rnd * s_ref * r_ref, starts=pos)
            ref_gpu_s += gs
            drift.append({"round": rnd, "dF": float(res["dF_JE"][-1]), "se": float(res["se_JE"][-1]), "gpu_s": gs})
        if rr is not None:
            rr.close()
        last = drift[-n_avg:] if n_avg else []
        F_ref = float(np.mean([d["dF"] for d in last])) if last else math.nan
        se_ref = math.sqrt(sum(d["se"] ** 2 for d in last)) / n_avg if last else math.nan
        slope = float(np.polyfit(np.arange(n_avg), [d["dF"] for d in last], 1)[0]) if n_avg > 1 else 0.0
        print(json.dumps({"beads": n_beads, "reference": {"dF_JE": F_ref, "se": se_ref, "drift_kT_per_round": slope / kT,
                                                          "rounds": drift}}), flush=True)
        init = pmf.pack_mlp_params(inputs.mlp_init_params(2))
        protocols = args.protocols
        rows = {k: [] for k in protocols}

        def continued(s_win, n_steps, seed):
            """s_win uniform windows for n_steps, then every replica continued
            from its end state for n_steps more (fresh uids); the estimate is
            the second run's, the GPU time both runs'."""
            res, gs1, rr = uniform(s_win, R, n_steps, seed)
            pos, _ = rr.final_state()
            rr.close()
            res, gs2, rr = uniform(s_win, R, n_steps, seed, uid_base=s_win * R, starts=pos)
            rr.close()
            return res, gs1 + gs2

        for seed in ([] if args.reference_only else aw["seeds"]):
            for tau in sorted(set(aw["tau_ps"]) | set(aw["tau_uniform_extra"])):
                n_steps = steps_of(tau)
                line = {"seed": seed, "tau_ps": tau}
                if "uniform" in protocols:
                    res, gs, rr = uniform(aw["s_uniform"], R, n_steps, seed)
                    rr.close()
                    rows["uniform"].append({"seed": seed, "tau_ps": tau, "gpu_s": gs, "windows": aw["s_uniform"],
                                            "dF": float(res["dF_JE"][-1]), "se": float(res["se_JE"][-1])})
                    line["uniform"] = rows["uniform"][-1]
                if tau not in aw["tau_ps"]:
                    print(json.dumps(line), flush=True)
                    continue
                for name, s_win in (("uniform_continued", aw["s_uniform"]), ("coarse_continued", aw["s_adaptive0"])):
                    if name in protocols:
                        res, gs = continued(s_win, n_steps, seed)
                        rows[name].append({"seed": seed, "tau_ps": tau, "gpu_s": gs, "windows": s_win,
                                           "dF": float(res["dF_JE"][-1]), "se": float(res["se_JE"][-1])})
                        line[name] = rows[name][-1]
                if "adaptive" not in protocols:
                    print(json.dumps(line), flush=True)
                    continue
                run.replicas, run.n_steps, run.n_equil, run.seed = R, n_steps, n_steps // 10, seed
                lam0 = np.linspace(aw["lo"], aw["hi"], aw["s_adaptive0"])
                meta, ares = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.3,
                                                  max_rounds=args.adaptive_rounds, max_windows=81, mlp_steps=400,
                                                  mlp_batch=512, mlp_lr=3e-3, mlp_seed=5 + seed,
                                                  continue_windows=not args.no_continuation,
                                                  train_on_gap=not args.no_train_gate)
                rows["adaptive"].append({"seed": seed, "tau_ps": tau, "gpu_s": meta["gpu_seconds"],
                                         "windows": meta["n_windows"], "rounds": meta["rounds"],
                                         "dF": float(ares["dF_JE"][-1]), "se": float(ares["se_JE"][-1])})
                line["adaptive"] = rows["adaptive"][-1]
                print(json.dumps(line), flush=True)

        def summary(rs):
            return ladder_summary(rs, aw["seeds"], F_ref, kT)

        out["chains"].append({"beads": n_beads, "lambda": [aw["lo"], aw["hi"]], "kT": kT, "replicas": R,
                              "adaptive_rounds": args.adaptive_rounds, "continuation": not args.no_continuation,
                              "train_gate": not args.no_train_gate,
                              "reference": {"dF_JE": F_ref, "se": se_ref, "drift_kT_per_round": slope / kT,
                                            "averaged_rounds": n_avg, "gpu_s": ref_gpu_s, "windows": s_ref,
                                            "replicas": r_ref, "md_steps_per_round": tau_ref, "rounds": drift},
                              **{k: summary(v) for k, v in rows.items()}, "runs": rows})
        sysh.close()
        print(json.dumps(out["chains"][-1]), flush=True)
    print(json.dumps(out), flush=True)


def _od1d_exact(lams, a, k, kT):
    """F(lambda, k) - F(lambda_1, k) of the 1D double well with its trap,
    -kT ln int exp(-(a (x^2 - 1)^2 + k/2 (x - lambda)^2) / kT) dx, by the
    trapezoid rule on a fine grid (the reference of the 1D ladder)."""
    x = np.linspace(-4.0, 4.0, 400001)
    U = a * (x * x - 1.0) ** 2
    F = []
    for lam in lams:
        e = -(U + 0.5 * k * (x - lam) ** 2) / kT
        m = e.max()
        F.append(-kT * (m + np.log(np.trapezoid(np.exp(e - m), x))))
    F = np.array(F)
    return F - F[0]


def bench_adaptive_1d(args, pmf, torch):
    """The GPU-seconds-to-0.2-kT comparison on the 1D double well, whose
    reference is exact (quadrature): the uniform 21-window grid against the
    learned placement from 11 windows (the chain study's protocol settings),
    32 replicas per window, a ladder of window lengths, seeds 0..4."""
    from paper_1105_4840_gb300 import inputs

    w = inputs.od1d_workload()
    run = w["run"]
    kT = run.kT
    lo, hi = float(run.lambdas[0]), float(run.lambdas[-1])
    exact = float(_od1d_exact([lo, hi], w["a"], run.k, kT)[-1])
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    init = pmf.pack_mlp_params(inputs.mlp_init_params(2))
    ladder = [250, 500, 1000, 2000, 4000, 8000, 16000, 32000]
    seeds = list(args.seeds) if args.seeds else [0, 1, 2, 3, 4]
    rows = {"uniform": [], "adaptive": []}
    for seed in seeds:
        for n_steps in ladder:
            run.replicas, run.n_steps, run.n_equil, run.seed, run.stride = 32, n_steps, n_steps // 10, seed, 10
            lam = np.linspace(lo, hi, 21)
            rr = pmf.pmf_run_prepare(sysh, lam, pmf.make_params(run))
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record()
            rr.launch()
            rr.reduce()
            ev[1].record()
            rr.wait()
            torch.cuda.synchronize()
            res = rr.free_energy()
            rr.close()
            rows["uniform"].append({"seed": seed, "steps": n_steps, "gpu_s": ev[0].elapsed_time(ev[1]) / 1000.0,
                                    "windows": 21, "dF": float(res["dF_JE"][-1])})
            meta, ares = pmf.pmf_run_adaptive(sysh, np.linspace(lo, hi, 11), pmf.make_params(run), init,
                                              threshold=0.3, max_rounds=3, max_windows=81, mlp_steps=400,
                                              mlp_batch=512, mlp_lr=3e-3, mlp_seed=5 + seed,
                                              continue_windows=not args.no_continuation,
                                              train_on_gap=not args.no_train_gate)
            rows["adaptive"].append({"seed": seed, "steps": n_steps, "gpu_s": meta["gpu_seconds"],
                                     "windows": meta["n_windows"], "rounds": meta["rounds"],
                                     "dF": float(ares["dF_JE"][-1])})

    def summary(rs):
        per_seed = []
        for seed in seeds:
            lad = sorted([r for r in rs if r["seed"] == seed], key=lambda r: r["steps"])
            ok = [abs(r["dF"] - exact) < 0.2 * kT for r in lad]
            first = next((i for i in range(len(lad)) if all(ok[i:])), None)
            per_seed.append(None if first is None else {"steps": lad[first]["steps"], "gpu_s": lad[first]["gpu_s"]})
        got = [x["gpu_s"] for x in per_seed if x is not None]
        by_steps = {}
        for n in ladder:
            dev = [r["dF"] - exact for r in rs if r["steps"] == n]
            by_steps[n] = {"mean_dev_kT": float(np.mean(dev)) / kT, "sd_dev_kT": float(np.std(dev)) / kT,
                           "mean_gpu_s": float(np.mean([r["gpu_s"] for r in rs if r["steps"] == n]))}
        return {"median_gpu_s": statistics.median(got) if got else None, "seeds_converged": len(got),
                "per_seed": per_seed, "by_steps": by_steps}

    out = {"workload": "od1d_adaptive_vs_uniform", "criterion_kT": 0.2, "lambda": [lo, hi],
           "exact_dF": exact, "replicas": 32, "dt": run.dt, "continuation": not args.no_continuation,
           "train_gate": not args.no_train_gate,
           "uniform": summary(rows["uniform"]), "adaptive": summary(rows["adaptive"]), "runs": rows}
    sysh.close()
    print(json.dumps(out), flush=True)


def bench_mlp(args, pmf, torch, stream):
    """Surrogate training throughput: Adam steps of the 1 -> 64 -> 64 -> 2
    network (64 x 64 layer on tcgen05, BF16 operands, FP32 accumulators in
    TMEM) on mini-batches drawn from a 1D run's sample store, split (a CTA
    per 128-sample tile, then an update launch, per step) and in one CTA."""
    from paper_1105_4840_gb300 import inputs

    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    lam = run.lambdas
    batch, steps = args.mlp_batch, args.mlp_steps
    tiles = (batch + 127) // 128
    flops = steps * tiles * 3 * 2 * 128 * 64 * 64  # Z2, dH1, dW2 of the 64 x 64 layer
    peak = float(_peaks().get("bf16_tflops", 1939.8))
    lines = {}
    for split in (1, 0):
        mlp = pmf.Mlp(pmf.pack_mlp_params(inputs.mlp_init_params(2)), 0.5 * (lam[0] + lam[-1]),
                      0.5 * (lam[-1] - lam[0]))
        mlp.set_split(split)
        for _ in range(args.warmup):
            mlp.train(rr, 50, batch, 3e-3, 1)
        times = []
        for i in range(args.steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            loss = mlp.train(rr, steps, batch, 3e-3, 100 + i)
            e[1].record(stream)
            torch.cuda.synchronize()
            times.append(e[0].elapsed_time(e[1]) / 1000.0)
        t = statistics.median(times)
        lines[split] = {"value": steps / t, "us_per_step": 1e6 * t / steps, "samples_per_s": steps * batch / t,
                        "loss": loss, "ctas": tiles if split else 1,
                        "tensor_tflops": flops / t / 1e12, "tensor_frac": flops / t / 1e12 / peak}
        mlp.close()
    line = {"workload": "surrogate_training", "metric": "adam_steps/s", "value": lines[1]["value"], "unit": "steps/s",
            "batch": batch, "steps_per_launch": steps, "split": lines[1], "one_cta": lines[0],
            "tensor_peak_tflops": peak, "note": "latency bound: a 4418-parameter network, 4 tiles per step"}
    print(json.dumps(line), flush=True)


def bench_spp(args, pmf, torch, stream):
    """Sequential pulling protocol on the 104-bead chain: `--replicas`
    independent simulations (672 by default, the parallel workload's count)
    each visit the 21 windows in order, `--md-steps` steps per window."""
    w = _workload(args.md_steps)
    p, start, run = w["params"], w["start"], w["run"]
    run.replicas = args.replicas
    sysh = pmf.pmf_create_system_chain([p], [start])
    rr = pmf.pmf_run_prepare_sequential(sysh, run.lambdas, pmf.make_params(run))
    for _ in range(args.warmup):
        rr.launch()
        rr.wait()
    sim_ms, red_ms = [], []
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.5)
    for _ in range(args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(stream)
        rr.launch()
        e[1].record(stream)
        rr.reduce()
        e[2].record(stream)
        torch.cuda.synchronize()
        sim_ms.append(e[0].elapsed_time(e[1]))
        red_ms.append(e[1].elapsed_time(e[2]))
    clocks.stop()
    rr.wait()
    res = rr.free_energy()
    steps = run.replicas * run.lambdas.size * run.n_steps
    t = statistics.mean(a + b for a, b in zip(sim_ms, red_ms))
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sm_count * 128 * 2 * float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved = steps * flops_per_replica_step(N_BEADS) / (statistics.mean(sim_ms) / 1000.0) / 1e12
    clk = clocks.summary()
    warps, ctas, seg = pmf.pmf_chain_get_launch(sysh, 0)
    line = {"workload": "chain104_spp", "metric": "replica-steps/s", "value": steps / (t / 1000.0),
            "unit": "replica-steps/s", "ms_per_step": t, "steps": args.steps, "warmup": args.warmup,
            "config": {"simulations": run.replicas, "windows": int(run.lambdas.size),
                       "md_steps_per_window": run.n_steps, "warps_per_replica": warps,
                       "launch": f"persistent, {'auto' if ctas == 0 else ctas} CTAs, segments <= {seg} steps"},
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons")},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak},
            "dF_JE_end": float(res["dF_JE"][-1]), "se_JE_end": float(res["se_JE"][-1]),
            "dF_fluct_end": float(res["dF_fluct"][-1])}
    print(json.dumps(line), flush=True)


def bench_histograms(args, pmf, torch, stream):
    """App. C work distributions on the 104-bead workload's samples with the
    paper's bins (dx = 0.001 A, dW = 0.01 kcal/mol, W in +-150 kcal/mol),
    after a PPP run of --md-steps steps per window."""
    w = _workload(args.md_steps)
    p, start, run = w["params"], w["start"], w["run"]
    sysh = pmf.pmf_create_system_chain([p], [start])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    dx, K = 1e-4, 50000                      # 0.001 A bins over 0..5 nm
    dw = 0.01 * 4.184                        # 0.01 kcal/mol in kJ/mol
    M = int(round(150 * 4.184 / dw))         # +-150 kcal/mol
    for _ in range(args.warmup):
        rr.work_distributions(0.0, dx, K, dw, M, with_omega=False)
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = rr.work_distributions(0.0, dx, K, dw, M, with_omega=False)
        times.append(time.perf_counter() - t0)
    res = rr.free_energy()
    line = {"workload": "chain104_app_c_histograms", "metric": "ms", "value": 1000 * statistics.median(times),
            "unit": "ms per call (host wall clock, synchronous)", "x_bins": K, "w_bins": 2 * M + 1,
            "samples": int(run.lambdas.size * run.replicas * ((run.n_steps - run.n_equil) // run.stride)),
            "dF_JE_end_hist": float(g["dF_JE"][-1]), "dF_JE_end_factorised": float(res["dF_JE"][-1]),
            "lost_max": float(g["lost"].max())}
    print(json.dumps(line), flush=True)


def bench_sweeps(args, pmf, torch, stream):
    """The experiments of Sec. IV B-D on the 104-bead chain: the 21-window
    run's estimates from every second window (s = 11), a spring-constant sweep
    and a relaxation-time sweep, with the wall time of each run."""
    from paper_1105_4840_gb300 import sweeps

    w = _workload(args.md_steps)
    p, start, run = w["params"], w["start"], w["run"]
    sysh = pmf.pmf_create_system_chain([p], [start])
    lam = run.lambdas
    t0 = time.perf_counter()
    rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
    full = rr.free_energy()
    t_full = time.perf_counter() - t0
    sub = sweeps.subsample(rr, lam, run.k, run.kT, every=2)
    ks = sweeps.k_sweep(sysh, lam, run, [100.0, 500.0, 2500.0])
    taus = sweeps.tau_sweep(sysh, lam, run, [int(t / run.dt) for t in (50.0, 100.0, 200.0, 400.0, 800.0)],
                            at_lambda=2.6)
    kT = run.kT
    line = {"workload": "chain104_sweeps", "kT": kT, "md_steps_per_window": run.n_steps,
            "delta_lambda": {"s21": {"dF_JE": float(full["dF_JE"][-1]), "dF_fluct": float(full["dF_fluct"][-1]),
                                     "seconds": t_full},
                             "s11": {"dF_JE": float(sub["dF_JE"][-1]), "dF_fluct": float(sub["dF_fluct"][-1])}},
            "k_sweep": [{"k": o["k"], "dF_JE": float(o["result"]["dF_JE"][-1]),
                         "dF_fluct": float(o["result"]["dF_fluct"][-1]),
                         "min_dF_fluct": float(o["result"]["dF_fluct"].min()),
                         "gamma2_mean": float(np.mean(o["result"]["gamma2"])), "seconds": o["seconds"]} for o in ks],
            "tau_sweep": taus}
    print(json.dumps(line), flush=True)


def bench_smd(args, pmf, torch, stream):
    """Constant-velocity pulling of the 104-bead chain from 1.3 to 3.3 nm:
    `--replicas` trajectories (672 by default), 10 % of `--md-steps` at the
    start position, then the trap moves 2 nm over the remaining steps."""
    w = _workload(args.md_steps)
    p, start, run = w["params"], w["start"], w["run"]
    run.replicas = args.replicas
    run.n_equil = run.n_steps // 10
    v = 2.0 / ((run.n_steps - run.n_equil) * run.dt)  # nm / ps
    sysh = pmf.pmf_create_system_chain([p], [start])
    rr = pmf.pmf_run_prepare_smd(sysh, 1.3, v, pmf.make_params(run))
    for _ in range(args.warmup):
        rr.launch()
        rr.wait()
    times = []
    for _ in range(args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        e[0].record(stream)
        rr.launch()
        e[1].record(stream)
        torch.cuda.synchronize()
        times.append(e[0].elapsed_time(e[1]))
    rr.wait()
    res = rr.smd_free_energy()
    steps = run.replicas * run.n_steps
    t = statistics.mean(times)
    line = {"workload": "chain104_smd", "metric": "replica-steps/s", "value": steps / (t / 1000.0),
            "unit": "replica-steps/s", "ms_per_step": t, "trajectories": run.replicas, "md_steps": run.n_steps,
            "velocity_nm_per_ns": v * 1000.0, "lambda_end": float(res["lambda"][-1]),
            "dF_JE_end": float(res["dF_JE"][-1]), "dF_cumulant_end": float(res["dF_cumulant"][-1]),
            "W_mean_end": float(res["W_mean"][-1]), "W_sd_end": float(math.sqrt(res["W_var"][-1]))}
    print(json.dumps(line), flush=True)


def od1d_cpu_baseline(w):
    """The FP64 oracle on the whole 1D workload (cpu_baseline leg), one thread
    per core over the replicas."""
    import concurrent.futures as cf

    from oracle import _clib

    run = w["run"]
    cores = os.cpu_count() or 1
    jobs = [(i, r) for i in range(run.lambdas.size) for r in range(run.replicas)]

    def one(job):
        i, r = job
        _clib.od1d_run(w["a"], run.lambdas[i], run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil,
                       run.stride, run.seed, i * run.replicas + r, w["x0"])

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, jobs))
    el = time.perf_counter() - t0
    return {"value": len(jobs) * run.n_steps / el, "unit": "replica-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole 1D workload ({len(jobs)} replicas x {run.n_steps} steps, FP64, {el:.2f} s)"}


def bench_od1d(args, pmf, torch, stream):
    """The 1D double-well workload (21 windows x 8 replicas x 2e4 steps,
    FP64): the whole PPP and its reductions per timed step."""
    from paper_1105_4840_gb300 import inputs

    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_prepare(sysh, run.lambdas, pmf.make_params(run))
    for _ in range(args.warmup):
        rr.launch()
        rr.reduce()
        rr.wait()
    times = []
    for _ in range(args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        e[0].record(stream)
        rr.launch()
        rr.reduce()
        e[1].record(stream)
        torch.cuda.synchronize()
        times.append(e[0].elapsed_time(e[1]))
    rr.wait()
    res = rr.free_energy()
    t = statistics.median(times)
    steps = run.lambdas.size * run.replicas * run.n_steps
    line = {"workload": "od1d_ppp", "metric": "replica-steps/s", "value": steps / (t / 1000.0),
            "unit": "replica-steps/s", "ms_per_step": t, "dtype": "f64", "windows": int(run.lambdas.size),
            "replicas_per_window": run.replicas, "md_steps_per_window": run.n_steps,
            "dF_JE_end": float(res["dF_JE"][-1]), "dF_JE_min": float(res["dF_JE"].min())}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = od1d_cpu_baseline(w)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--md-steps", type=int, default=400000, help="BAOAB steps per window (workload: 4e5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="chain104",
                    choices=["chain104", "batch64", "precision", "adaptive", "mlp", "spp", "histograms", "sweeps",
                             "smd", "od1d", "adaptive1d"],
                    help="chain104: the 104-bead PPP (default); batch64: 64 uneven chains in one graph; "
                         "precision: FP32 vs FP64 integration study")
    ap.add_argument("--replicas", type=int, default=1024, help="replicas per window (precision study)")
    ap.add_argument("--mlp-steps", type=int, default=2000, help="Adam steps per timed launch (mlp)")
    ap.add_argument("--mlp-batch", type=int, default=512, help="mini-batch (mlp)")
    ap.add_argument("--adaptive-beads", type=int, nargs="+", default=[104, 200], help="chain lengths (adaptive)")
    ap.add_argument("--reference-steps", type=int, default=None,
                    help="steps per window and round of the continued reference (adaptive; default 0.4 ns)")
    ap.add_argument("--reference-rounds", type=int, default=None,
                    help="rounds of the continued reference (adaptive; 0: none)")
    ap.add_argument("--reference-average", type=int, default=None, help="last reference rounds averaged")
    ap.add_argument("--reference-only", action="store_true", help="adaptive: run the reference alone")
    ap.add_argument("--protocols", nargs="+", default=["uniform", "adaptive"],
                    choices=["uniform", "adaptive", "uniform_continued", "coarse_continued"],
                    help="adaptive: protocols to run (the continued ones run tau twice, the second run estimating)")
    ap.add_argument("--reference-replicas", type=int, default=None, help="replicas per reference window")
    ap.add_argument("--adaptive-replicas", type=int, default=None, help="replicas per window (adaptive)")
    ap.add_argument("--tau-uniform-extra", type=float, nargs="*", default=None,
                    help="relaxation times run by the uniform grid only (adaptive)")
    ap.add_argument("--adaptive-rounds", type=int, default=2, help="insertion rounds of the learned placement")
    ap.add_argument("--no-continuation", action="store_true",
                    help="learned placement: later rounds run the inserted windows only")
    ap.add_argument("--no-train-gate", action="store_true",
                    help="learned placement: train in every round, even without a measured overlap gap")
    ap.add_argument("--tau-ps", type=float, nargs="+", default=None, help="relaxation-time ladder (adaptive)")
    ap.add_argument("--seeds", type=int, nargs="+", default=None, help="dynamics seeds (adaptive)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from __graft_entry__ import build

    if rank == 0 or world == 1:
        build()
    if dist is not None:
        dist.barrier()
    from paper_1105_4840_gb300 import pmf

    stream = torch.cuda.current_stream()
    pmf.pmf_set_stream(stream.cuda_stream)
    if args.workload == "batch64":
        if world == 1:
            bench_batch(args, pmf, torch, stream)
        return
    if args.workload == "od1d":
        if world == 1:
            bench_od1d(args, pmf, torch, stream)
        return
    if args.workload == "smd":
        if world == 1:
            if args.replicas == 1024:
                args.replicas = 672
            bench_smd(args, pmf, torch, stream)
        return
    if args.workload == "sweeps":
        if world == 1:
            bench_sweeps(args, pmf, torch, stream)
        return
    if args.workload == "histograms":
        if world == 1:
            bench_histograms(args, pmf, torch, stream)
        return
    if args.workload == "spp":
        if world == 1:
            if args.replicas == 1024:  # the precision study's default is not meant here
                args.replicas = 672
            bench_spp(args, pmf, torch, stream)
        return
    if args.workload == "mlp":
        if world == 1:
            bench_mlp(args, pmf, torch, stream)
        return
    if args.workload == "adaptive":
        if world == 1:
            bench_adaptive(args, pmf, torch)
        return
    if args.workload == "adaptive1d":
        if world == 1:
            bench_adaptive_1d(args, pmf, torch)
        return
    if args.workload == "precision":
        if world == 1:
            bench_precision(args, pmf, torch)
        return
    w = _workload(args.md_steps)
    p, start, run = w["params"], w["start"], w["run"]
    s, R = run.lambdas.size, run.replicas
    n_rep = s * R
    from paper_1105_4840_gb300.shard import shard_uid_base

    uid_base = shard_uid_base(rank, s, R)
    sysh = pmf.pmf_create_system_chain([p], [start])
    # untimed setup: pick warps per replica from short probes of this run
    warps, _ = pmf.pmf_chain_autotune(sysh, run.lambdas, pmf.make_params(run, uid_base=uid_base), probe_steps=10000)
    _, grid_ctas, seg_steps = pmf.pmf_chain_get_launch(sysh, 0)
    rr = pmf.pmf_run_prepare(sysh, run.lambdas, pmf.make_params(run, uid_base=uid_base))
    replica_steps = n_rep * run.n_steps
    chunks = math.ceil(run.n_steps / 100000)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    from paper_1105_4840_gb300 import shard

    def one_step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        rr.launch()
        if ev is not None:
            ev[1].record(stream)
        if dist is None:
            rr.reduce()
        else:
            # the exchange step: every rank's per-replica partials, merged
            rr.wait()
            merged = shard.gather_partials(rr.partials(), device=torch.device("cuda", local))
            pmf.pmf_free_energy_from_partials(merged, run.lambdas, run.k, run.kT)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        one_step()
    torch.cuda.synchronize()
    rr.wait()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    _nvtx(torch, "timed")  # lets a profiler capture exactly the timed launches
    for i in range(args.steps):
        flush.fill_(float(i))  # L2 flush (256 MB) between timed steps, outside the events
        one_step(evs[i])
    torch.cuda.synchronize()
    _nvtx(torch, None)
    if dist is not None:
        dist.barrier()
    clocks.stop()
    rr.wait()
    res = rr.free_energy()
    sim_ms = [e[0].elapsed_time(e[1]) for e in evs]
    red_ms = [e[1].elapsed_time(e[2]) for e in evs]
    step_ms = [a + b for a, b in zip(sim_ms, red_ms)]
    t_step = sum(step_ms) / len(step_ms)
    if dist is not None:
        t = torch.tensor([t_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    value = world * replica_steps / (t_step / 1000.0)

    # end to end through the C ABI with host buffers: system upload, run, results
    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sys2 = pmf.pmf_create_system_chain([p], [start])
        pmf.pmf_chain_set_warps(sys2, 0, warps)
        pmf.pmf_chain_set_grid(sys2, 0, grid_ctas, seg_steps)
        r2 = pmf.pmf_run_windows(sys2, run.lambdas, pmf.make_params(run, uid_base=uid_base))
        out = r2.free_energy()
        e2e_times.append(time.perf_counter() - t0)
        h2d = 8 * (p.n * 7 + p.n * 6 + p.n * 3) + 4 + 8 * s * 1 + 8 * 4 * s
        d2h = 8 * len(out) * s + 4
        r2.close()
        sys2.close()
    e2e_value = world * replica_steps / statistics.median(e2e_times)
    # after the timed region: the measured FP32 FMA rate of this GPU (scalar
    # and packed f32x2), the practical ceiling beside the derived peak
    ffma2_tflops, _ = pmf.pmf_fp32_peak(packed=True)
    ffma_tflops, _ = pmf.pmf_fp32_peak(packed=False)
    dfma_tflops, _ = pmf.pmf_fp64_peak()

    if rank != 0:
        return
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    clk = clocks.summary()
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    chain_launch_ms = sum(sim_ms) / (len(sim_ms) * chunks)
    flops_launch = n_rep * min(run.n_steps, 100000) * flops_per_replica_step(N_BEADS)
    achieved = flops_launch / (chain_launch_ms / 1000.0) / 1e12
    traffic = _ncu_traffic(warps)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops,
            "traffic": (traffic or {}).get("dram_bytes_per_launch"),
            "kernel": f"chain_kernel<float,{warps}>",
            "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)",
            "frac_at_sampled_clock": (achieved / (sm_count * 256 * clk["sm_mhz"] * 1e6 / 1e12)
                                      if clk.get("sm_mhz") else None),
            "flops_per_replica_step": flops_per_replica_step(N_BEADS),
            "launch_ms": chain_launch_ms,
            "peak_measured": {"ffma2": ffma2_tflops, "ffma": ffma_tflops, "unit": "TFLOP/s",
                              "source": "pmf_fp32_peak: 8 independent FMA chains per thread, 4 x 512 threads per SM"},
            "frac_of_measured": achieved / max(ffma2_tflops, ffma_tflops)}
    ns_per_day = replica_steps * world / (t_step / 1000.0) * run.dt * 86400.0 / 1e3
    line = {"metric": "replica-steps/s", "value": value, "unit": "replica-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(run, world),
            "launch": {"warps_per_replica": warps, "ctas": "auto" if grid_ctas == 0 else grid_ctas,
                       "segment_steps": seg_steps, "mode": "persistent",
                       "schedule_variant": pmf.pmf_chain_get_schedule(sysh, 0)},
            "e2e": {"value": e2e_value, "unit": "replica-steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * (chunks + 3),
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons")},
            "roofline": roof,
            "aggregate_ns_per_day": ns_per_day,
            "reduction_ms": sum(red_ms) / len(red_ms),
            "reduction": _reduction_roofline(sum(red_ms) / len(red_ms), n_rep * world * samples_per_replica(run),
                                             peaks, dfma_tflops),
            "dF_JE_end": float(res["dF_JE"][-1]), "dF_fluct_end": float(res["dF_fluct"][-1]),
            "dF_com_end": float(res["dF_com"][-1]), "uncertainty_end": float(res["uncertainty"][-1])}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
