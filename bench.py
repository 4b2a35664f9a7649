"""Benchmark: effective sparse-grid points per second of Smolyak quadrature
on one GB300 (or N independent replicas under torchrun).

Workload (default): d = 12, Gauss-Legendre rule (level l has l nodes),
q = d + 6, Genz oscillatory integrand with seeded parameters, FP64; one step
= one integral (table setup, item values, the persistent fold kernel and the
fixed-order reduction).  The metric's unit is n_d^q, the point count of
Eq. 2.6 with repetition (593,775 here).

--impl reference times the CPU oracle (the plain enumeration the tests use
as ground truth) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective sparse-grid points/sec and s/integral at stated rel. error vs FP64 oracle"


# DRAM bytes per launch of the timed fold kernel, from the ncu capture
# summarised in profiles/sg_fold_kernel_d__cfg2_d12_gl_L6_oscillatory.txt.
# Valid only for the kernel sources with this digest; otherwise reported as
# null until the capture is taken again.
_FOLD_TRAFFIC = {"cfg2_d12_gl_L6_oscillatory": (290304, "9a83459e18b4fae8")}
_KERNEL_SOURCES = ["paper_2210_14313_gb300/csrc/sg_kernels.cu", "paper_2210_14313_gb300/csrc/sg_fold_logic.h",
                   "paper_2210_14313_gb300/csrc/sg_ff.cuh", "paper_2210_14313_gb300/csrc/sg_internal.h",
                   "paper_2210_14313_gb300/csrc/sg_reduce.cuh", "paper_2210_14313_gb300/csrc/sg_fixed.h",
                   "paper_2210_14313_gb300/csrc/sg_xsum.h"]


def _kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for p in _KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _fold_traffic(name, prec):
    t = _FOLD_TRAFFIC.get(name)
    if t is None or prec != 0 or t[1] != _kernel_digest():
        return None
    return t[0]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(name):
    import sg_inputs as si
    if name == "cfg2":
        return si.cfg2(), 0
    if name == "cfg3":
        return si.cfg3(si.FAM_GAUSSIAN), 1
    if name == "cfg5":
        return si.cfg5(), 0
    if name == "cfg1":
        return si.cfg1(), 0
    raise SystemExit("unknown workload " + name)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_rate(c, budget_s=12.0):
    """Oracle throughput (points/s) on this host, repeated up to a time budget."""
    import oracle
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 200:
            break
    dt = time.perf_counter() - t0
    pts = oracle.count_points(c["rule"], c["d"], c["L"])
    return pts * n / dt, n, dt


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the job's timed region ends with its
    slowest rank); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    c, _prec = _workload(args.workload)
    oracle.build()
    pts = oracle.count_points(c["rule"], c["d"], c["L"])
    for _ in range(args.warmup):
        oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    cores = os.cpu_count()
    value = pts * len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": c["name"], "d": c["d"], "q": c["d"] + c["L"], "rule": "gauss_legendre"
                   if c["rule"] == 4 else "clenshaw_curtis", "points_per_integral": pts,
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": "%d whole integrals of the workload" % len(times)},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_gpu(args):
    import numpy as np
    import torch
    import paper_2210_14313_gb300 as sg
    import oracle

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c, prec = _workload(args.workload)
    if args.prec is not None:
        prec = {"fp64": 0, "mixed": 1, "ff": 2}[args.prec]
    d, L = c["d"], c["L"]
    q = d + L
    rule = sg.Rule(c["rule"], max_level=L + 1)
    pts, evals = sg.count_points(rule, d, q)
    stream = torch.cuda.current_stream()
    dparams = torch.tensor(c["params"], dtype=torch.float64, device="cuda")
    dout = torch.zeros(sg.DEV_RESULT_DOUBLES, dtype=torch.float64, device="cuda")
    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        sg.integrate_async(rule, c["fam"], dparams, d, q, dout, prec=prec)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # accuracy of the timed configuration against the oracle
    ref = oracle.integrate(c["rule"], c["fam"], c["params"], d, L)
    got = dout.cpu().numpy()
    rel_err = abs(got[0] * 2.0 ** (got[1] - ref.exp2) - ref.mant) / abs(ref.mant)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sg.profile_begin(stream)
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    fold_ms, fold_launches = sg.profile_end(stream)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot_ms = max_over_ranks(sum(ms), dist, torch.device("cuda", local))
    value = ws * pts * args.steps / (tot_ms * 1e-3)

    # end to end through the public blocking call, host buffers (pinned)
    hparams = torch.tensor(c["params"], dtype=torch.float64).pin_memory()
    hp = hparams.numpy()
    for _ in range(3):
        sg.integrate(rule, c["fam"], hp, d, q, prec=prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(args.steps, 5)
    for _ in range(ne):
        sg.integrate(rule, c["fam"], hp, d, q, prec=prec)
    e2e_s = (time.perf_counter() - t0) / ne
    e2e = {"value": ws * pts / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(hparams.numel() * 8),
           "d2h_bytes_per_step": 56, "s_per_integral": e2e_s}

    # roofline of the fold kernel against the measured per-point ceiling
    fold_avg_s = fold_ms * 1e-3 / max(fold_launches, 1)
    achieved = evals / fold_avg_s
    kind = 1 if c["fam"] == 1 else 0
    peak = sg.ceiling(prec, kind)
    fma_peak = sg.ceiling(prec, 2)

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f64", 1: "f32-eval/f64-sum", 2: "f32x2-eval/f64-sum"}[prec],
        "data": "synthetic (seeded SplitMix64 parameters)",
        "config": {"workload": c["name"], "d": d, "q": q,
                   "rule": {1: "trapezoid", 2: "clenshaw_curtis", 4: "gauss_legendre"}[c["rule"]],
                   "family": sg_family_name(c["fam"]), "points_per_integral": pts,
                   "evals_per_integral": evals, "form": "telescoped",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "flushed between steps (256 MB write)",
                   "rel_err_vs_oracle": rel_err},
        "s_per_integral": tot_ms * 1e-3 / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gevals/s",
                     "frac": achieved / peak, "traffic": _fold_traffic(c["name"], prec),
                     "peak_source": "measured per-point ceiling kernel (sg_ceiling), same run",
                     "fma_peak_tflops": fma_peak / 1e12},
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,  # setup + fold per integral
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_extra:
        line["extra"] = _extras(sg, oracle, torch)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        oracle.build()
        rate, n, dt = _oracle_rate(c)
        line["cpu_baseline"] = {"value": rate, "unit": "points/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": "%d whole integrals in %.1f s" % (n, dt)}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def _extras(sg, oracle, torch):
    """Precision ladder on every configuration and a batch subset (one GPU):
    seconds per integral and relative error against the oracle."""
    import numpy as np
    import sg_inputs as si
    rules = {k: sg.Rule(k, max_level=8) for k in (2, 4)}
    out = {"configs": {}, "batch": {}}
    names = {0: "fp64", 1: "mixed", 2: "ff"}
    for c in [si.cfg1(), si.cfg2(), si.cfg3(si.FAM_PRODUCT_PEAK), si.cfg3(si.FAM_GAUSSIAN), si.cfg5()]:
        ref = oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
        row = {"points": oracle.count_points(c["rule"], c["d"], c["L"])}
        for prec in (0, 1, 2):
            ts = []
            for _ in range(7):
                r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=prec)
                ts.append(r.seconds)
            t = sorted(ts)[3]
            err = abs(r.mant * 2.0 ** (r.exp2 - ref.exp2) - ref.mant) / abs(ref.mant)
            row[names[prec]] = {"s_per_integral": t, "points_per_s": row["points"] / t, "rel_err": err,
                                "err_est": r.err_est}
        out["configs"][c["name"]] = row
    # batch subset: the first items of the 4096-item workload whose point
    # count stays below 5e9 (so that the FP64 form finishes in seconds)
    items = [it for it in si.batch()[:1200]
             if oracle.count_points(it["rule"], it["d"], it["L"]) <= 5e9][:96]
    specs, pool, off = [], [], 0
    for it in items:
        specs.append((rules[it["rule"]], it["fam"], it["d"], it["d"] + it["L"], off))
        pool.append(np.asarray(it["params"]))
        off += 2 * it["d"]
    pool = np.concatenate(pool)
    pts = sum(oracle.count_points(it["rule"], it["d"], it["L"]) for it in items)
    small = [k for k, it in enumerate(items)
             if oracle.count_points(it["rule"], it["d"], it["L"]) <= 5e6][:24]
    refs = [oracle.integrate(items[k]["rule"], items[k]["fam"], items[k]["params"], items[k]["d"],
                             items[k]["L"]) for k in small]
    out["batch"]["items"] = len(items)
    out["batch"]["points"] = pts
    for label, prec, g in (("fp64", 0, 0.0), ("mixed", 1, 0.0), ("mixed_guard_ff_1e-6", 1, 2.5e-7), ("ff", 2, 0.0)):
        sg.integrate_batch(specs, pool, prec=prec, guard_tol=g)
        res = sg.integrate_batch(specs, pool, prec=prec, guard_tol=g)
        t = res[0].seconds
        errs = [abs(res[k].mant * 2.0 ** (res[k].exp2 - o.exp2) - o.mant) / abs(o.mant)
                for k, o in zip(small, refs)]
        out["batch"][label] = {"s": t, "points_per_s": pts / t,
                               "max_rel_err_vs_oracle": max(errs) if errs else None,
                               "oracle_checked_items": len(errs),
                               "max_err_est": max(r.err_est for r in res)}
    return out


def sg_family_name(f):
    return {0: "exp_linear", 1: "oscillatory", 2: "product_peak", 3: "gaussian", 4: "gaussian_lin"}[f]


def _sweep_params(fam, d):
    """The integrands of Test 10 (Section 6.2) on [0,1]^d as library families."""
    import numpy as np
    if fam == "f1":  # exp(sum (-1)^(i+1) x_i)
        return 0, np.concatenate([[(-1.0) ** i for i in range(d)], np.zeros(d)])
    if fam == "f2":  # prod 1 / (0.9^2 + (x_i - 0.6)^2)
        return 2, np.concatenate([np.full(d, 1 / 0.9), np.full(d, 0.6)])
    if fam == "f3":  # exp(-|x|^2 / 2) (the constant factor does not change the work)
        return 3, np.concatenate([np.full(d, math.sqrt(0.5)), np.zeros(d)])
    # f4: cos(2 pi + sum x_i)
    return 1, np.concatenate([np.ones(d), [1.0], np.zeros(d - 1)])


def _fit(xs, ts):
    """Least-squares t = c x^b on log scales: (b, c, R^2)."""
    import numpy as np
    lx, lt = np.log(np.asarray(xs, float)), np.log(np.asarray(ts, float))
    b, a = np.polyfit(lx, lt, 1)
    pred = a + b * lx
    ss = float(((lt - pred) ** 2).sum()), float(((lt - lt.mean()) ** 2).sum())
    return float(b), float(math.exp(a)), 1.0 - ss[0] / ss[1] if ss[1] > 0 else 1.0


def run_sweep(args):
    """Section 6's complexity experiment on the GPU: the time of one integral
    against the dimension d at fixed excess levels L = 2, 3, 4 (and at d = 10
    for more levels) for the Test 10 integrands, three rules (Clenshaw-Curtis,
    Gauss-Legendre, Gauss-Patterson with the accuracy-level growth) and two
    precisions.  One JSON line per measurement (median of 5 blocking calls),
    then the power-law fits t = c d^b over the runs well above the launch
    floor and the fits t = t0 + evals / R (launch floor and rate)."""
    import numpy as np
    import torch
    import paper_2210_14313_gb300 as sg
    torch.cuda.set_device(0)
    rules = {"cc": sg.Rule(sg.RULE_CLENSHAW_CURTIS, max_level=10),
             "gl": sg.Rule(sg.RULE_GAUSS_LEGENDRE, max_level=10),
             "gp": sg.Rule(sg.RULE_GAUSS_PATTERSON, max_level=13, growth=sg.GROWTH_SLOW)}
    budget = float(args.sweep_budget)
    series, rates = {}, {}
    ds = [5, 10, 20, 50, 100, 200, 500, 1000, 2000]
    for rname, rule in rules.items():
        for fam in ("f1", "f2", "f3", "f4"):
            for prec in (sg.PREC_FP64, sg.PREC_MIXED):
                runs = [(L, d) for L in (2, 3, 4) for d in ds] + [(L, 10) for L in (1, 5, 6, 7, 8)]
                for L, d in runs:
                    pts, ev = sg.count_points(rule, d, d + L)
                    if ev > budget * (1 if prec == sg.PREC_FP64 else 20):
                        continue
                    f, p = _sweep_params(fam, d)
                    for _ in range(2):
                        sg.integrate(rule, f, p, d, d + L, prec=prec)
                    t = sorted(sg.integrate(rule, f, p, d, d + L, prec=prec).seconds for _ in range(5))[2]
                    rec = {"sweep": "complexity", "rule": rname, "integrand": fam,
                           "prec": {0: "fp64", 1: "mixed"}[prec], "d": d, "L": L, "points": pts,
                           "evals": ev, "s": t, "points_per_s": pts / t}
                    print(json.dumps(rec), flush=True)
                    series.setdefault((rname, fam, rec["prec"], L), []).append((d, t))
                    rates.setdefault((rname, fam, rec["prec"]), []).append((ev, t))
    for (rname, fam, prec, L), pts in sorted(series.items()):
        # power law in d over the runs well above the launch floor
        floor = min(t for _, t in pts)
        use = [(x, t) for x, t in pts if t >= 5 * floor]
        if len(use) < 3:
            use = sorted(pts)[-3:]
        if len(use) < 3:
            continue
        b, c, r2 = _fit([x for x, _ in use], [t for _, t in use])
        print(json.dumps({"fit": "t = c d^b", "rule": rname, "integrand": fam, "prec": prec, "L": L,
                          "b": round(b, 3), "c": c, "r2": round(r2, 4),
                          "range": [min(x for x, _ in use), max(x for x, _ in use)]}), flush=True)
    for (rname, fam, prec), pts in sorted(rates.items()):
        # t = t0 + evals / R over all runs (least squares)
        e = np.asarray([x for x, _ in pts], float)
        t = np.asarray([y for _, y in pts], float)
        inv_r, t0 = np.polyfit(e, t, 1)
        print(json.dumps({"fit": "t = t0 + evals / R", "rule": rname, "integrand": fam, "prec": prec,
                          "t0_us": round(t0 * 1e6, 1), "R_evals_per_s": 1.0 / inv_r if inv_r > 0 else None,
                          "runs": len(pts)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--prec", default=None, choices=[None, "fp64", "mixed", "ff"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="run the complexity sweep of Section 6 instead of the benchmark")
    ap.add_argument("--sweep-budget", default="4e9", help="largest FP64 evaluation count per run")
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
