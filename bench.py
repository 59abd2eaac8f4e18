#!/usr/bin/env python
"""Throughput of the GB300 TT-cross quadrature on the D_12 workload.

A step is one whole integral: the initial index set, then sweeps of the
dimension-parallel cross (new core entries, QR of the cross matrices,
contraction, Alg. 2 on every interface, set update) until a stopping rule
fires.  The workload is D_12 in R^12 (trapezoid on [-24, 24], 385 nodes per
mode, rank cap 64, tol 1e-12, seed 12); the problem's node tables stay
resident in HBM across steps and L2 is flushed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload d12|c4|e16]

One JSON line on rank 0.  Under torchrun every rank runs its own replica of the
workload on its own GPU (the path does not shard: replicas only, weak scaling).
"""
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

METRIC = "integrals/s & fiber evals/s at rel.err<=1e-12 vs plain sweep; p50/p99 latency"
# DRAM bytes (read + write) per launch of the kernels the roofline may name,
# from one ncu capture each (plain launches of this bench on the
# D_12 workload); null for a kernel whose code changed after its capture
NCU_TRAFFIC = {"k_solve": {"bytes_per_launch": 859733, "capture": "profiles/k_solve_d12.md: launches 301-303 "
                           "(sweep ~50), dram__bytes_read.sum + dram__bytes_write.sum"}}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
KERNELS = ("eval_slabs", "qr", "contract", "samples", "rook_col", "rook_row", "update", "init", "setup",
           "solve", "search")


def workload(name):
    from paper_1903_11554_gb300 import inputs
    return {"d12": inputs.config_d12, "c4": inputs.config_c4, "e16": inputs.config_e16,
            "d12_r4": inputs.config_d12_r4, "d12_p4": inputs.config_d12_p4,
            "d8": lambda: inputs.config_d_cube(8), "d32": lambda: inputs.config_d_cube(32)}[name]()


def workload_config(p):
    return {"workload": "%s: %s_%d, %s form, N=%d/mode, d=%d, rank cap %d, tol %g, %s contraction, seed %d"
            % (p.name, p.family, p.n, "R^n trapezoid" if p.form == "rn" else "unit-cube Gauss-Legendre",
               p.N[0], p.d, p.rank_cap, p.tol, p.precision, p.seed)
            + (", up to %d pivots per interface per sweep" % p.npiv if p.npiv > 1 else ""),
            "family": p.family, "n": p.n, "d": p.d, "nodes_per_mode": p.N[0], "rank_cap": p.rank_cap,
            "tol": p.tol, "precision": p.precision, "l2": "flushed between steps (256 MB write)"}


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", "oracle_full.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    return g.get(name)


# --------------------------------------------------------------------------
# clocks sampled during the timed region

class Clocks:
    def __init__(self, index):
        self.path = tempfile.mktemp(prefix="ttq_clk_", suffix=".csv")
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # start before the timed region: wait for the sampler's first lines
            t0 = time.time()
            while time.time() - t0 < 10.0:
                self.f.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.05)
            time.sleep(0.5)
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
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        load = [v for v in sm if v > 0.5 * mx] or sm
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# --------------------------------------------------------------------------
# CPU baseline: the oracle, timed on a bounded sample of the workload
#
# A sample is a set of whole sweeps of the workload's stored oracle run
# (tests/golden/oracle_full.json), spread evenly over its sweep range
# (stratified: sweep s_q = floor((q + 1/2) S / K) of S, q = 0..K-1).  Each
# sampled sweep starts from that run's own index sets at that sweep (the first
# r_k(s) rows of its final nested sets: pivots are appended in order, so a
# prefix is the state of an earlier sweep) and runs exactly as the oracle's
# integrate() runs it: every core re-evaluated, the integral contracted, Alg. 2
# on every interface, the pivots appended.  The K sweeps stand for K / S of an
# integral, so integrals/s = (K / S) / (their summed wall time).  Every number
# is a timed measurement; nothing is fitted or extrapolated.

SWEEP_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import ttcross
from paper_1903_11554_gb300 import inputs
p = {"d12": inputs.config_d12, "c4": inputs.config_c4, "e16": inputs.config_e16}[%(wl)r]()
g = json.load(open(os.path.join(%(root)r, "tests", "golden", "oracle_full.json")))[%(wl)r]
ranks_at = g["history_ranks"]
par = g["parents"]
out = []
for s in %(sweeps)r:
    rk = ranks_at[s]
    lp = [np.array(par["lpar"][k - 1][:rk[k]]) for k in range(1, p.d)]
    ln = [np.array(par["lnode"][k - 1][:rk[k]]) for k in range(1, p.d)]
    rp = [np.array(par["rpar"][k - 1][:rk[k]]) for k in range(1, p.d)]
    rn = [np.array(par["rnode"][k - 1][:rk[k]]) for k in range(1, p.d)]
    st = ttcross.from_parents(p, lp, ln, rp, rn)
    assert st.ranks() == rk
    t = time.perf_counter()
    value, cores, scale, piv = ttcross.sweep(p, st, s, search=s < len(ranks_at) - 1)
    st = ttcross.apply_pivots(p, st, piv)
    dt = time.perf_counter() - t
    out.append([s, max(rk), dt, abs(value / float(g["history"][s]) - 1.0)])
    print(json.dumps(out[-1]), flush=True)
"""


def stratified(total, k):
    """Sweep indices of a stratified sample of k sweeps of a total-sweep run
    (with repeats when k > total, so the sample still stands for k / total of it)."""
    return [min(total - 1, int((q + 0.5) * total / k)) for q in range(k)]


def cpu_info():
    model = ""
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"host_cpus": os.cpu_count(), "cpu_model": model or "unknown"}


def oracle_sweeps(wl, sweeps, threads, timeout):
    """Time the given sweeps of the workload's stored oracle run in a fresh
    process (the oracle never shares a process with the GPU path); threads =
    BLAS threads (the oracle's integrand evaluation is single-threaded numpy)."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    code = SWEEP_SNIPPET % {"root": ROOT, "wl": wl, "sweeps": list(sweeps)}
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
    rows = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("[")]
    if len(rows) != len(sweeps):
        raise RuntimeError("oracle sweep timing failed: %s" % out.stderr[-2000:])
    return rows


def cpu_baseline(wl, k_sweeps=3):
    """The oracle on one host core and on all of them (BLAS threads), each on
    the same stratified sample of k_sweeps sweeps of the workload."""
    g = golden(wl)
    total = g["sweeps"]
    sw = stratified(total, k_sweeps)
    info = cpu_info()
    res = {}
    for label, th in (("one_core", 1), ("all_cores", info["host_cpus"] or 1)):
        rows = oracle_sweeps(wl, sw, th, timeout=1800)
        secs = sum(r[2] for r in rows)
        res[label] = {"value": (len(rows) / total) / secs, "cores": th, "seconds": round(secs, 2),
                      "sweeps_timed": [r[0] for r in rows], "ranks": [r[1] for r in rows],
                      "max_rel_diff_vs_stored_run": max(r[3] for r in rows)}
    one = res["one_core"]
    return {"value": one["value"], "unit": "integrals/s", "cores": 1, "kind": "oracle",
            "sample": "oracle sweeps %s of the %d-sweep %s run (ranks %s), each from that run's own index sets at that "
                      "sweep, timed on one host core in %.1f s; they stand for %d/%d of an integral (stratified "
                      "sample, no fit)" % (one["sweeps_timed"], total, wl, one["ranks"], one["seconds"],
                                           len(one["sweeps_timed"]), total),
            "max_rel_diff_vs_stored_run": one["max_rel_diff_vs_stored_run"], "all_cores": res["all_cores"], **info}


# --------------------------------------------------------------------------

def measure_eval_full(plan, p, flush, reps=3):
    """Kernel (a) on every entry of the final cores: the run's final index sets
    are set back on the plan (so every fiber counts as new) and one sweep runs
    without pivot search; CUDA events around the evaluation launch and its
    device FP64 counter give its achieved rate.  Best of `reps`."""
    st = plan.get_state()
    ranks = st["ranks"]
    entries = sum(ranks[k - 1] * p.N[k - 1] * ranks[k] for k in range(1, p.d + 1))
    best = None
    for _ in range(reps):
        plan.set_state(ranks, st["lpar"], st["lnode"], st["rpar"], st["rnode"])
        flush.zero_()
        plan.set_timing(True)
        plan.kernel_times(reset=True)
        plan.sweep(0, search=False)
        kt = plan.kernel_times()["eval_slabs"]
        plan.set_timing(False)
        tf = kt["flops"] / (kt["ms"] / 1000.0) / 1e12 if kt["ms"] > 0 else 0.0
        if best is None or kt["ms"] < best["ms"]:
            best = {"ms": kt["ms"], "tflops": tf}
    return {"kernel": "k_eval_slabs", "entries": entries, "ms": best["ms"],
            "entries_per_s": entries / (best["ms"] / 1000.0), "achieved_tflops": best["tflops"],
            "peak_tflops": FP64_PEAK_TFLOPS, "frac": best["tflops"] / FP64_PEAK_TFLOPS,
            "note": "one launch evaluating every entry of the final D_12 cores (ranks %s), best of %d" % (
                max(ranks), reps)}


def measure_workload(binding, torch, name, steps, flush):
    """Another configured workload (C_4 or E_16), timed like the headline one:
    warm-up runs, then `steps` whole integrals enqueued back to back on the
    plan's stream with the L2 flushed between them, CUDA events around them;
    its error against the stored oracle run, and the oracle's own time on the
    host (C_4: whole integrals on one core; E_16: a stratified two-sweep sample)."""
    p = workload(name)
    plan = binding.Plan(p)
    stream = plan.stream
    for q in range(3):
        with torch.cuda.stream(stream):
            flush.zero_()
        plan.launch(q)
    for q in range(3):
        plan.result(q)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        plan.launch(q % 64)
    e1.record(stream)
    torch.cuda.synchronize()
    res = [plan.result(q) for q in range(min(steps, 64))]
    ms = e0.elapsed_time(e1)
    plan.close()
    out = {"workload": workload_config(p)["workload"], "integrals_per_s": steps / (ms / 1000.0),
           "ms_per_integral": ms / steps, "fiber_evals_per_s": res[-1]["n_eval"] * steps / (ms / 1000.0),
           "value": res[-1]["value"], "value_lo": res[-1]["value_lo"], "status": res[-1]["status_name"],
           "sweeps": res[-1]["sweeps"], "max_rank": res[-1]["max_rank"], "n_eval": res[-1]["n_eval"],
           "runs_identical": all(r == res[0] for r in res)}
    g = golden(name)
    if g is not None:
        ref = float(g["value"])
        out["rel_err_vs_oracle"] = abs(res[-1]["value"] - ref) / abs(ref)
        if "value_exact_contraction" in g:
            ex = float(g["value_exact_contraction"])
            out["rel_err_vs_oracle_cores_at_60_digits"] = abs(res[-1]["value"] + res[-1]["value_lo"] - ex) / abs(ex)
        out["same_trajectory_as_oracle"] = (res[-1]["sweeps"], res[-1]["n_eval"]) == (g["sweeps"], g["n_eval"])
        if name in ("d12_r4", "d12_p4", "d8"):
            pass
        elif name == "c4":
            env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
            code = ("import sys, time, json; sys.path.insert(0, %r)\n"
                    "from oracle import ttcross\nfrom paper_1903_11554_gb300 import inputs\n"
                    "p = inputs.config_c4(); ttcross.integrate(p)\n"
                    "t = time.perf_counter(); n = 0\n"
                    "while time.perf_counter() - t < 5.0:\n    ttcross.integrate(p); n += 1\n"
                    "print(json.dumps([n, time.perf_counter() - t]))" % ROOT)
            o = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
            n, secs = json.loads(o.stdout.strip().splitlines()[-1])
            out["cpu_oracle"] = {"value": n / secs, "unit": "integrals/s", "cores": 1,
                                 "sample": "%d whole C_4 oracle integrals in %.1f s on one host core" % (n, secs)}
        elif "history_ranks" in g:
            rows = oracle_sweeps(name, stratified(g["sweeps"], 2), 1, timeout=1800)
            secs = sum(r[2] for r in rows)
            out["cpu_oracle"] = {"value": (len(rows) / g["sweeps"]) / secs, "unit": "integrals/s", "cores": 1,
                                 "sample": "oracle sweeps %s of the %d-sweep run on one host core, %.1f s; they stand "
                                           "for %d/%d of an integral" % ([r[0] for r in rows], g["sweeps"], secs,
                                                                         len(rows), g["sweeps"])}
    if name == "c4":
        # the closed form C_4 = 7 zeta(3) / 12; zeta(3) by the series
        # (5/2) sum_n (-1)^(n+1) / (n^3 binom(2n, n)), whose terms fall ~4x per n
        z3 = 2.5 * math.fsum((-1) ** (n + 1) / (n ** 3 * math.comb(2 * n, n)) for n in range(1, 40))
        ref = 7.0 * z3 / 12.0
        out["closed_form"] = {"value": ref, "formula": "7 zeta(3) / 12",
                              "rel_err": abs(res[-1]["value"] - ref) / ref,
                              "note": "rank cap 16 and the truncated trapezoid grid limit this run, not the arithmetic"}
    printed = paper_value(name)
    if printed is not None:
        out["rel_err_vs_printed_value"] = abs(res[-1]["value"] + res[-1]["value_lo"] - printed["value"]) / printed["value"]
        out["printed_value"] = printed
    return out


def paper_value(name):
    """The paper's printed value of a workload (tests/golden/paper_values.json), if any."""
    key = {"d8": "D_8", "d32": "D_32"}.get(name)
    path = os.path.join(ROOT, "tests", "golden", "paper_values.json")
    if key is None or not os.path.exists(path):
        return None
    e = json.load(open(path))[key]
    return {"value": float(e["value"]), "source": e["source"]}


def measure_search_variants(binding, torch, flush, steps=3):
    """D_12 with the search as one persistent kernel per sweep (same results bit
    for bit as the staged launches, timed the same way), and with the
    sequential sweep of Alg. 5 (another algorithm: its value beside Alg. 6's)."""
    p = workload("d12")
    out = {}
    for label in ("persistent_search", "sequential_alg5"):
        plan = binding.Plan(p)
        if label == "persistent_search":
            plan.set_search(True)
        else:
            plan.set_sequential(True)
        ref = plan.run()
        torch.cuda.synchronize()
        n = steps if label == "persistent_search" else 1
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(plan.stream)
        res = []
        for _ in range(n):
            with torch.cuda.stream(plan.stream):
                flush.zero_()
            res.append(plan.run())
        t1.record(plan.stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / n
        out[label] = {"integrals_per_s": 1000.0 / ms, "ms_per_integral": ms, "value": res[-1]["value"],
                      "sweeps": res[-1]["sweeps"], "n_eval": res[-1]["n_eval"], "status": res[-1]["status_name"],
                      "runs_identical": all(r == ref for r in res)}
        plan.close()
    return out


def measure_batched(binding, inputs, torch, count=256):
    """The 256-instance mixed batch (families C/D/E cyclic, n in 4..24, N in
    {65,129,257,513}, rank caps in {8..128}): autotuned, one warm-up run, one
    timed run; then the same 256 problems one at a time (a plan each, its
    second run timed), results compared bit for bit; and the batch's error
    against the stored oracle runs of 24 of its instances."""
    probs = inputs.batched_mix(count)
    b = binding.Batch(probs)
    tuned = b.autotune(2)
    b.run()
    torch.cuda.synchronize()
    t = time.time()
    res = b.run()
    dt = time.time() - t
    del b
    torch.cuda.empty_cache()
    st, same = 0.0, True
    for q in range(count):
        pl = binding.Plan(probs[q])
        pl.run()
        torch.cuda.synchronize()
        t = time.time()
        r = pl.run()
        st += time.time() - t
        same &= (r == res[q])
        pl.close()
    errs = {}
    path = os.path.join(ROOT, "tests", "golden", "batch_oracle.json")
    if os.path.exists(path):
        for key, ref in json.load(open(path)).items():
            errs[key] = abs(res[int(key)]["value"] - float(ref["value"])) / abs(float(ref["value"]))
    return {"workload": "%d mixed instances (C/D/E cyclic, n 4..24, N 65..513, rank cap 8..128, tol 1e-12, "
                        "seed 256+i)" % count,
            "integrals_per_s": count / dt, "seconds": dt, "autotuned": tuned,
            "concurrent_groups": min(8, max(1, count // 32)),
            "statuses": {k: sum(1 for r in res if r["status_name"] == k) for k in set(r["status_name"] for r in res)},
            "fiber_evals_per_s": sum(r["n_eval"] for r in res) / dt,
            "one_at_a_time": {"integrals_per_s": count / st, "seconds": st,
                              "results_identical_to_batch": bool(same)},
            "batched_over_one_at_a_time": (count / dt) / (count / st),
            "rel_err_vs_oracle": {"instances": len(errs), "max": max(errs.values()) if errs else None}}


def measure_serving(binding, inputs, torch, count=2000, rate=2000.0, pool_gb=120.0, max_slots=1024,
                    sweeps_per_step=2, alone=0, batched=False):
    """Poisson arrivals (rate per second, seeded), families uniform over C/D/E,
    n in 4..32, tol log-uniform in [1e-14, 1e-8], N in {129, 257, 513}, rank cap
    64; HBM admission budget pool_gb; sweeps_per_step sweeps of every request
    in flight per server step.  Latency = completion seen by the host minus
    scheduled arrival.  alone > 0: the first `alone` requests of the same
    stream are also run one at a time (a plan each over one workspace: upload,
    whole run, result read back), for the served-against-alone rate."""
    arrivals, probs = inputs.serving_stream(count, rate)
    pool_bytes = int(pool_gb * (1 << 30))
    srv = binding.Server(pool_bytes, max_slots=max_slots)
    srv.set_mode(batched)
    t0 = time.time()
    i, lat, when, ids = 0, {}, {}, {}
    peak_flight, peak_queue = 0, 0
    results = {}
    while len(results) < count:
        now = time.time() - t0
        while i < count and arrivals[i] <= now:
            rid = srv.submit(probs[i])
            ids[rid] = i
            when[rid] = arrivals[i]
            i += 1
        flight, queued, _ = srv.step(sweeps_per_step)
        peak_flight = max(peak_flight, flight)
        peak_queue = max(peak_queue, queued)
        done = srv.drain()
        tnow = time.time() - t0
        for rid, r in done.items():
            results[rid] = r
            lat[rid] = tnow - when[rid]
        if flight == 0 and queued == 0 and i < count and not done:
            time.sleep(max(0.0, min(0.01, arrivals[i] - (time.time() - t0))))
    span = time.time() - t0
    srv.close()
    del srv
    torch.cuda.empty_cache()
    ls = sorted(lat.values())
    # a few served results against the same problem run alone
    same = True
    for rid in list(results)[:8]:
        same &= (binding.integrate(probs[ids[rid]]) == results[rid])
    out = {"workload": "Poisson %g req/s, %d requests (seed 2000), C/D/E, n 4..32, tol 1e-14..1e-8, N 129..513, "
                       "rank cap 64, HBM admission budget %g GB, %s"
                       % (rate, count, pool_gb, ("batched engine, %d sweeps per server step" % sweeps_per_step)
                          if batched else "concurrent engine (a plan and graph per request, 16 streams)"),
           "offered_per_s": count / float(arrivals[-1]), "achieved_integrals_per_s": count / span,
           "latency_s": {"p50": ls[len(ls) // 2], "p99": ls[min(len(ls) - 1, int(math.ceil(0.99 * len(ls))) - 1)]},
           "peak_in_flight": peak_flight, "peak_queued": peak_queue, "seconds": span,
           "served_equal_alone_on_8": bool(same)}
    if alone > 0:
        ws = torch.empty(max(binding.workspace_bytes(p) for p in probs[:alone]), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        t = time.time()
        for p in probs[:alone]:
            pl = binding.Plan(p, workspace=ws)
            pl.run()
            pl.close()
        torch.cuda.synchronize()
        secs = time.time() - t
        out["one_at_a_time"] = {"requests": alone, "integrals_per_s": alone / secs, "seconds": secs}
        out["served_over_one_at_a_time"] = (count / span) / (alone / secs)
    return out


def max_over_ranks(x, dist, device):
    """The largest of a per-rank quantity over the process group (the slowest
    rank sets the job's time); x itself when there is one process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units every rank processed over the job's time."""
    return units_per_rank * world / (ms / 1000.0)


def run_reference(args):
    """The reference arm: the oracle as it stands, on the host's cores (BLAS
    threads = all of them), on the same workload.  A step is one whole sweep of
    the workload's stored oracle run; the W warm-up steps are its first W sweeps,
    the K timed steps a stratified sample of K sweeps (see cpu_baseline), so the
    timed steps stand for K / S of an integral."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = workload(args.workload)
    g = golden(args.workload)
    total = g["sweeps"]
    info = cpu_info()
    threads = info["host_cpus"] or 1
    warm = list(range(min(args.warmup, total)))
    timed_sweeps = stratified(total, args.steps)
    rows = oracle_sweeps(args.workload, warm + timed_sweeps, threads, timeout=7200)
    timed = rows[len(warm):]
    secs = sum(r[2] for r in timed)
    v = (len(timed) / total) / secs
    sample = ("%d whole sweeps of the %d-sweep oracle run of the workload (stratified: sweeps %s, ranks up to %d), "
              "each from that run's own index sets at that sweep, %.1f s in all on %d host threads (BLAS); they stand "
              "for %d/%d of an integral; %d warm-up sweeps before them"
              % (len(timed), total, [r[0] for r in timed], max(r[1] for r in timed), secs, threads, len(timed), total,
                 len(warm)))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "integrals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(p),
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": v, "unit": "integrals/s",
                             "max_rel_diff_vs_stored_run": max(r[3] for r in timed), **info},
            "e2e": {"value": v, "unit": "integrals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="d12", choices=["d12", "c4", "e16"])
    ap.add_argument("--cpu-sweeps", type=int, default=2, help="oracle sweeps in the cpu_baseline sample")
    ap.add_argument("--no-systems", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--launch-mode", default="graph", choices=["graph", "plain"],
                    help="graph: one CUDA graph per integral (default); plain: every kernel a stream launch")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1903_11554_gb300 import binding, build, inputs
    if rank == 0:
        build.build()
    barrier()
    build.build()
    p = workload(args.workload)
    plan = binding.Plan(p)
    plan.set_graphs(args.launch_mode == "graph")
    stream = plan.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    nwarm = max(3, args.warmup)
    for q in range(nwarm):                   # warm up the same path the timed region uses
        with torch.cuda.stream(stream):
            flush.zero_()
        plan.launch(q % 64)
    for q in range(nwarm):
        plan.result(q % 64)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident, K whole integrals (per-sweep CUDA graph)
    l0 = plan.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    results = []
    lat = []
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        # K whole integrals enqueued back to back on the plan's stream (one graph
        # each); the L2 flush runs on the same stream between them
        for q in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.launch(q % 64)
            b.record(stream)
            lat.append((a, b))
            if q % 64 == 63:
                results.extend(plan.result(s) for s in range(64))
        e1.record(stream)
        torch.cuda.synchronize()
        results.extend(plan.result(s) for s in range(args.steps % 64))
        barrier()
    ms = e0.elapsed_time(e1)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    launches = plan.launches - l0
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_rate(args.steps, world, ms)
    n_eval = sum(r["n_eval"] for r in results)
    evals_per_s = job_rate(n_eval, world, ms)

    # ---- per-kernel device time (CUDA events around every launch on its stream)
    # and algorithmic FP64 operations, over ROOF_STEPS more whole integrals
    ROOF_STEPS = 2
    plan.set_timing(True)
    plan.kernel_times(reset=True)
    k0 = plan.kernel_times()
    for _ in range(ROOF_STEPS):
        flush.zero_()
        plan.run()
    k1 = plan.kernel_times()
    plan.set_timing(False)
    kt = {}
    for name in KERNELS:
        kt[name] = {"ms": k1[name]["ms"] - k0[name]["ms"], "launches": k1[name]["launches"] - k0[name]["launches"],
                    "flops": k1[name]["flops"] - k0[name]["flops"]}
    if kt["search"]["launches"]:
        # the persistent search's FP64 operations are counted by stage
        kt["search"]["flops"] = sum(kt[n]["flops"] for n in ("samples", "rook_col", "rook_row", "solve"))
    side = {"contract"}                                  # runs on the side stream, beside the search
    main = {k: v for k, v in kt.items() if k not in side and v["launches"]}
    dom = max(main, key=lambda n: main[n]["ms"])
    d = kt[dom]
    achieved = d["flops"] / (d["ms"] / 1000.0) / 1e12 if d["ms"] > 0 else 0.0
    tr = NCU_TRAFFIC.get("k_" + dom)
    roof = {"kernel": "k_" + dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": tr["bytes_per_launch"] if tr else None,
            "traffic_source": tr["capture"] if tr else None,
            "peak_source": "FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz "
                           "(nominal 1.25 TFLOP/s)",
            "algorithmic_flops_per_launch": d["flops"] / max(1, d["launches"]),
            "avg_launch_ms": d["ms"] / max(1, d["launches"]),
            "time_share_main_stream": d["ms"] / max(1e-9, sum(v["ms"] for v in main.values())),
            "measured_over": "%d whole integrals after the timed region, events around every launch" % ROOF_STEPS,
            "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                            "tflops": (v["flops"] / (v["ms"] / 1000.0) / 1e12) if v["ms"] > 0 else 0.0}
                        for k, v in kt.items() if v["launches"]}}

    # ---- the whole integral's algorithmic FP64 operations (the device
    # counters over the ROOF_STEPS integrals above) against its graph-timed
    # duration: how much of the FP64 peak one integral uses end to end
    per_int_flops = sum(v["flops"] for n, v in kt.items() if n != "search") / ROOF_STEPS
    whole = per_int_flops / (ms / args.steps / 1000.0) / 1e12
    fp64_whole = {"algorithmic_flops_per_integral": per_int_flops, "tflops": whole, "peak": FP64_PEAK_TFLOPS,
                  "frac": whole / FP64_PEAK_TFLOPS,
                  "note": "every kernel's counted FP64 operations of one integral / the integral's graph-timed "
                          "duration (ms_per_step)"}

    # ---- kernel (a) on whole cores: the final index sets set back on the plan
    # (every fiber new), one sweep without search; the evaluation kernel alone
    eval_full = measure_eval_full(plan, p, flush)

    # ---- end to end through the C ABI with host buffers
    h2d0, d2h0 = 0, 0
    torch.cuda.synchronize()
    ws = plan.workspace
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 5))
    h2d = d2h = 0
    barrier()
    t_host = time.time()
    f0.record(stream)
    for _ in range(e2e_steps):
        flush.zero_()
        q = binding.Plan(p, workspace=ws, stream=stream)   # host nodes/weights -> device inside the call
        r = q.run()                                          # result read back to the host
        hb, db = q.transfer_bytes()
        h2d += hb
        d2h += db
        q.close()
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(max(f0.elapsed_time(f1), (time.time() - t_host) * 1000.0), dist, "cuda")
    e2e = {"value": job_rate(e2e_steps, world, e2e_ms), "unit": "integrals/s",
           "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps}

    others = {}
    if args.workload == "d12" and args.launch_mode == "graph":
        for name in ("c4", "e16", "d12_r4", "d12_p4", "d8", "d32"):
            others[name] = measure_workload(binding, torch, name, max(3, min(args.steps, 20)), flush)
        others["d12_search_variants"] = measure_search_variants(binding, torch, flush)
    systems = {}
    if not args.no_systems and args.launch_mode == "graph":
        del plan
        torch.cuda.empty_cache()
        systems["batched"] = measure_batched(binding, inputs, torch)
        systems["serving"] = measure_serving(binding, inputs, torch, count=args.serving_requests, alone=100)
        systems["serving_batched_engine"] = measure_serving(binding, inputs, torch, count=400, batched=True)
        # the same stream kind offered at 70% of the capacity just measured, so
        # its latencies are service times rather than queueing under overload
        cap_rate = 0.7 * systems["serving"]["achieved_integrals_per_s"]
        systems["serving_below_capacity"] = measure_serving(binding, inputs, torch, count=300, rate=cap_rate)
    if rank != 0:
        return 0
    g = golden(args.workload)
    check = {}
    if g is not None:
        ref = float(g["value"])
        check = {"oracle_value": ref, "rel_err_vs_oracle": abs(results[-1]["value"] - ref) / abs(ref),
                 "oracle_sweeps": g["sweeps"], "oracle_seconds": g.get("oracle_seconds")}
    g = golden(args.workload)
    cpu = cpu_baseline(args.workload, args.cpu_sweeps) if (g and "history_ranks" in g and args.cpu_sweeps > 0) \
        else None
    line = {
        "metric": METRIC, "value": value, "unit": "integrals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(p), launch_mode=args.launch_mode),
        "fiber_evals_per_s": evals_per_s,
        "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)]},
        "result": {"value": results[-1]["value"], "value_lo": results[-1]["value_lo"], "sweeps": results[-1]["sweeps"],
                   "max_rank": results[-1]["max_rank"], "status": results[-1]["status_name"],
                   "n_eval": results[-1]["n_eval"], "internal_conv": results[-1]["internal_conv"], **check},
        "roofline": roof, "fp64_whole_integral": fp64_whole, "eval_full_cores": eval_full, "cpu_baseline": cpu,
        "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(),
        **others,
        **systems,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
