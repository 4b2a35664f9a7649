"""Benchmark: effective sparse-grid points per second of Smolyak quadrature
on one GB300 (or N independent replicas under torchrun).

Workload (default): d = 12, Gauss-Legendre rule (level l has l nodes),
q = d + 6, Genz oscillatory integrand, FP64 -- the single-integral FP64
configuration the headline metric is quoted on; the other configurations
(d = 4 Clenshaw-Curtis, the d = 100 and d = 1000 mixed-precision ones, the
4096-item batch, the d = 1000 gradient) are reported under "extra" or with
--workload.  One step = R independent integrals of the workload (R = 1024 by
default, each with its own seeded parameter draw), each a full single-integral
call (table setup, item values, the persistent fold kernel and the
deterministic reduction), issued back to back on one stream.  The metric's
unit is n_d^q, the point count of Eq. 2.6 with repetition (593,775 here).
The configurations under "extra" are timed the same way (64 draws back to
back, inputs resident on the device), each beside the latency of one
blocking call with host parameters on an idle GPU ("s_isolated_call").

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
_FOLD_TRAFFIC = {"cfg2_d12_gl_L6_oscillatory": (396544, "5a40fb25d655a1e7")}
_KERNEL_SOURCES = ["paper_2210_14313_gb300/csrc/sg_kernels.cu", "paper_2210_14313_gb300/csrc/sg_fold_logic.h",
                   "paper_2210_14313_gb300/csrc/sg_ff.cuh", "paper_2210_14313_gb300/csrc/sg_internal.h",
                   "paper_2210_14313_gb300/csrc/sg_reduce.cuh", "paper_2210_14313_gb300/csrc/sg_fixed.h",
                   "paper_2210_14313_gb300/csrc/sg_xsum.h", "paper_2210_14313_gb300/csrc/sg_lacc.h"]


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
    table = {"cfg1": (si.cfg1, 0), "cfg2": (si.cfg2, 0), "cfg3": (lambda: si.cfg3(si.FAM_GAUSSIAN), 1),
             "cfg3peak": (lambda: si.cfg3(si.FAM_PRODUCT_PEAK), 1), "cfg5": (si.cfg5, 0)}
    if name not in table:
        raise SystemExit("unknown workload " + name)
    f, prec = table[name]
    return f(), prec


RULE_NAMES = {1: "trapezoid", 2: "clenshaw_curtis", 3: "gauss_patterson", 4: "gauss_legendre"}


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
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


def _oracle_rate(c, budget_s=12.0, nthreads=0):
    """Oracle throughput (points/s) on this host over whole integrals,
    repeated up to a time budget (at least 3): (median rate, runs, seconds)."""
    import oracle
    pts = oracle.count_points(c["rule"], c["d"], c["L"])
    t_start = time.perf_counter()
    rates = []
    while True:
        t0 = time.perf_counter()
        oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"], nthreads=nthreads)
        rates.append(pts / (time.perf_counter() - t0))
        if len(rates) >= 3 and (time.perf_counter() - t_start > budget_s or len(rates) >= 200):
            break
    rates.sort()
    return rates[len(rates) // 2], len(rates), time.perf_counter() - t_start


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the job's timed region ends with its
    slowest rank); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def _config(c, pts, evals, per_step, form):
    return {"workload": c["name"], "d": c["d"], "q": c["d"] + c["L"], "rule": RULE_NAMES[c["rule"]],
            "family": sg_family_name(c["fam"]), "points_per_integral": pts, "evals_per_integral": evals,
            "integrals_per_step": per_step, "form": form,
            "inputs": "seeded parameter draws of the workload, one per integral (draw 0 = the "
                      "workload's own)",
            "l2": "flushed between steps (256 MB write); a step's integrals share the L2-resident plan"}


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
    cfg = _config(c, pts, pts, 1, "difference form, every point evaluated from the full d-vector")
    cfg["l2"] = "n/a (CPU)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": "one whole integral of the workload per step (draw 0)"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _fold_roofline(sg, prec, kind, pts, evals, fold_ms, launches):
    """Roofline of the fold kernel: effective points (the metric's unit) and
    evaluations per second against the measured per-point ceiling."""
    fold_avg_s = fold_ms * 1e-3 / max(launches, 1)
    peak = sg.ceiling(prec, kind)
    return {"bound": "alu", "achieved": pts / fold_avg_s / 1e9, "peak": peak / 1e9, "unit": "Gpoints/s",
            "frac": pts / fold_avg_s / peak, "achieved_evals": evals / fold_avg_s / 1e9,
            "frac_evals": evals / fold_avg_s / peak, "fold_us": fold_avg_s * 1e6,
            "peak_source": "measured per-point ceiling kernel (sg_ceiling: the fold's per-point "
                           "sequence on register-resident data), same run"}


def run_batch(args):
    """The 4096-integral batch workload at the 1e-6 bar: one step is the whole
    batch in one persistent launch per precision tier (float evaluation; the
    items whose estimate exceeds 1e-6 / 4 again in float-float; what that
    still leaves above it in FP64), checked item by item against the separable
    pin.  Minutes per step (by default one timed step after one warm-up step):
    not part of the default run."""
    import numpy as np
    import torch
    import paper_2210_14313_gb300 as sg
    import sg_inputs as si
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import dp_pin

    torch.cuda.set_device(0)
    rules = {k: sg.Rule(k, max_level=8) for k in (2, 4)}
    items = si.batch()
    specs, pool, off = [], [], 0
    for it in items:
        specs.append((rules[it["rule"]], it["fam"], it["d"], it["d"] + it["L"], off))
        pool.append(np.asarray(it["params"]))
        off += 2 * it["d"]
    pool = torch.tensor(np.concatenate(pool), dtype=torch.float64, device="cuda")
    pts = 0
    for it in items:
        pts += sg.count_points(rules[it["rule"]], it["d"], it["d"] + it["L"])[0]
    tol = 2.5e-7
    clocks = ClockSampler(0)
    clocks.start()
    times, res = [], None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = sg.integrate_batch(specs, pool, prec=sg.PREC_MIXED, guard_tol=tol)
        if k >= args.warmup:
            times.append((res[0].seconds, time.perf_counter() - t0))
    clk = clocks.stop()
    worst = 0.0
    for it, r in zip(items, res):
        rel, ls = dp_pin.smolyak_value_f64(it["rule"], it["fam"], it["params"], it["d"], it["L"])
        if it["fam"] == si.FAM_OSCILLATORY:
            err = abs(r.value - rel) / abs(rel)
        else:
            err = abs(r.mant * math.exp(r.exp2 * math.log(2.0) - ls) - rel) / abs(rel)
        worst = max(worst, err)
    dev = sum(t for t, _ in times)
    line = {"metric": METRIC, "value": pts * len(times) / dev, "unit": "points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-eval/f64-sum",
            "data": "synthetic (seeded SplitMix64 parameters)",
            "config": {"workload": "cfg4_batch4096", "items": len(items), "points": pts,
                       "guard_tol": tol, "tiers": "float, float-float, FP64", "form": "merged"},
            "max_rel_err_vs_separable_pin": worst, "s_per_batch_wall": times[-1][1],
            "clocks": clk}
    print(json.dumps(line))


def run_gpu(args):
    import ctypes
    import numpy as np
    import torch
    import paper_2210_14313_gb300 as sg
    import oracle
    import sg_inputs as si

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
    R = args.per_step
    rule = sg.Rule(c["rule"], max_level=L + 1)
    pts, evals = sg.count_points(rule, d, q)
    lib = sg.load()
    stream = torch.cuda.current_stream()
    sh = ctypes.c_void_p(stream.cuda_stream)
    hpar = np.stack([si.redraw(c, j) for j in range(R)])
    dparams = torch.tensor(hpar, dtype=torch.float64, device="cuda")
    dout = torch.zeros((R, sg.DEV_RESULT_DOUBLES), dtype=torch.float64, device="cuda")
    calls = [(rule.handle, c["fam"], ctypes.c_void_p(dparams[j].data_ptr()), d, q, prec, sg.FORM_AUTO, sh,
              ctypes.c_void_p(dout[j].data_ptr())) for j in range(R)]
    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        f = lib.sg_integrate_async
        for a in calls:
            if f(*a) != 0:
                raise RuntimeError("sg_integrate_async failed")

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # accuracy of the timed configuration against the oracle (the first draws)
    got = dout.cpu().numpy()
    errs = []
    for j in range(min(R, 4)):
        ref = oracle.integrate(c["rule"], c["fam"], hpar[j], d, L)
        errs.append(abs(got[j, 0] * 2.0 ** (got[j, 1] - ref.exp2) - ref.mant) / abs(ref.mant))

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    # the fold kernel's own device time, from events around each fold launch
    # of one more step (outside the timed region: the events sit between the
    # setup and fold launches)
    flush.fill_(-1.0)
    sg.profile_begin(stream)
    step()
    fold_ms, fold_launches = sg.profile_end(stream)
    ms = [s_.elapsed_time(e) for s_, e in zip(starts, ends)]
    tot_ms = max_over_ranks(sum(ms), dist, torch.device("cuda", local))
    value = ws * R * pts * args.steps / (tot_ms * 1e-3)

    # end to end through the public blocking call, host buffers (pinned):
    # parameters from host memory, the result record read back on the host
    hp = torch.tensor(hpar, dtype=torch.float64).pin_memory().numpy()
    for j in range(min(R, 8)):
        sg.integrate(rule, c["fam"], hp[j], d, q, prec=prec)
    torch.cuda.synchronize()
    ne = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(ne):
        for j in range(R):
            sg.integrate(rule, c["fam"], hp[j], d, q, prec=prec)
    e2e_s = (time.perf_counter() - t0) / (ne * R)
    e2e = {"value": ws * pts / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(R * 2 * d * 8),
           "d2h_bytes_per_step": int(R * 7 * 8), "s_per_integral": e2e_s,
           "how": "sg_integrate (blocking) per integral, host parameters in pinned memory, "
                  "result record read on the host; %d steps" % ne}

    kind = 1 if c["fam"] == 1 else 0
    roof = _fold_roofline(sg, prec, kind, pts, evals, fold_ms, fold_launches)
    roof["traffic"] = _fold_traffic(c["name"], prec)
    roof["fma_peak_tflops"] = sg.ceiling(prec, 2) / 1e12
    form = "merged (Eq. 2.8: every distinct point once, with its merged weight)"
    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f64", 1: "f32-eval/f64-sum", 2: "f32x2-eval/f64-sum"}[prec],
        "data": "synthetic (seeded SplitMix64 parameters)",
        "config": _config(c, pts, evals, R, form),
        "s_per_integral": tot_ms * 1e-3 / (args.steps * R),
        # draw 0 is the workload as configured; the other draws' errors beside it
        "rel_err_vs_oracle": errs[0], "rel_err_other_draws": errs[1:],
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": 2 * R * args.steps,  # setup + fold per integral
        "clocks": clk,
    }
    line["config"]["parallelism"] = "replicas" if ws > 1 else "single"
    if clk.get("sm_mhz"):
        line["clocks"]["ms_per_step_x_mhz"] = line["ms_per_step"] * clk["sm_mhz"]
    if rank == 0 and ws == 1 and not args.no_extra:
        line["extra"] = _extras(sg, oracle, torch, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        oracle.build()
        rate, n, dt = _oracle_rate(c, budget_s=8.0)
        rate1, n1, dt1 = _oracle_rate(c, budget_s=8.0, nthreads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "median of %d whole integrals (draw 0) in %.1f s, all cores" % (n, dt),
                                "one_thread": {"value": rate1, "cores": 1,
                                               "sample": "median of %d whole integrals in %.1f s" % (n1, dt1)}}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def _rel(r, o):
    return abs(r.mant * 2.0 ** (r.exp2 - o.exp2) - o.mant) / abs(o.mant)


def _extras(sg, oracle, torch, args):
    """The other configurations on one GPU: the precision ladder with the
    fold's roofline, the gradient of the d = 1000 configuration, the batched
    form of the headline workload, and a subset of the 4096-item batch."""
    import ctypes
    import numpy as np
    import sg_inputs as si
    rules = {k: sg.Rule(k, max_level=8) for k in (2, 4)}
    out = {"configs": {}, "batch": {}}
    names = {0: "fp64", 1: "mixed", 2: "ff"}
    stream = torch.cuda.current_stream()
    for c in [si.cfg1(), si.cfg2(), si.cfg3(si.FAM_PRODUCT_PEAK), si.cfg3(si.FAM_GAUSSIAN), si.cfg5()]:
        ref = oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
        rule = rules[c["rule"]]
        row = {"points": oracle.count_points(c["rule"], c["d"], c["L"])}
        # R draws resident on the device, integrated back to back through the
        # asynchronous entry point (as the headline step), events around them;
        # and the latency of one blocking call with host parameters, GPU idle
        R = 64
        dpar = torch.tensor(np.stack([si.redraw(c, j) for j in range(R)]), dtype=torch.float64, device="cuda")
        dout = torch.zeros((R, sg.DEV_RESULT_DOUBLES), dtype=torch.float64, device="cuda")
        q = c["d"] + c["L"]
        lib = sg.load()
        sh = ctypes.c_void_p(stream.cuda_stream)
        for prec in (0, 1, 2):
            calls = [(rule.handle, c["fam"], ctypes.c_void_p(dpar[j].data_ptr()), c["d"], q, prec, sg.FORM_AUTO,
                      sh, ctypes.c_void_p(dout[j].data_ptr())) for j in range(R)]

            def run():
                for a in calls:
                    if lib.sg_integrate_async(*a) != 0:
                        raise RuntimeError("sg_integrate_async failed")
            for _ in range(3):
                run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            sg.profile_begin(stream)
            run()
            fold_ms, nl = sg.profile_end(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3 / R
            ts = []
            for _ in range(11):
                r = sg.integrate(rule, c["fam"], c["params"], c["d"], q, prec=prec)
                ts.append(r.seconds)
            rr = _fold_roofline(sg, prec, 1 if c["fam"] == 1 else 0, r.points, r.evals, fold_ms, nl)
            row[names[prec]] = {"s_per_integral": t, "points_per_s": row["points"] / t, "rel_err": _rel(r, ref),
                                "s_isolated_call": sorted(ts)[5],
                                "err_est": r.err_est, "evals": r.evals,
                                "roofline": {k: rr[k] for k in ("achieved", "peak", "frac", "frac_evals",
                                                                "fold_us")}}
        out["configs"][c["name"]] = row
    # the d = 1000 configuration with its gradient (2000 entries): forward
    # sum plus the adjoint sub-sums and the assembly kernel, through the
    # blocking call with host buffers
    c = si.cfg5()
    q = c["d"] + c["L"]
    for prec in (0, 1):
        for _ in range(2):
            sg.integrate_grad(rules[2], c["fam"], c["params"], c["d"], q, prec=prec)
        ts, walls = [], []
        for _ in range(7):
            t0 = time.perf_counter()
            r, g = sg.integrate_grad(rules[2], c["fam"], c["params"], c["d"], q, prec=prec)
            walls.append(time.perf_counter() - t0)
            ts.append(r.seconds)
        t, w = sorted(ts)[3], sorted(walls)[3]
        out["configs"].setdefault("cfg5_gradient", {})[names[prec]] = {
            "s_per_call": t, "s_per_call_wall": w, "points": r.points, "evals_incl_adjoint": r.evals,
            "evals_per_s": r.evals / t, "gradient_entries": int(g.size)}
    # the headline workload in the batched form: R draws in one persistent launch
    c = si.cfg2()
    R = min(args.per_step, 1024)
    specs, pool = [], []
    for j in range(R):
        specs.append((rules[4], c["fam"], c["d"], c["d"] + c["L"], 2 * c["d"] * j))
        pool.append(si.redraw(c, j))
    pool = np.concatenate(pool)
    for prec in (0, 1):
        sg.integrate_batch(specs, pool, prec=prec)
        res = sg.integrate_batch(specs, pool, prec=prec)
        o = oracle.integrate(c["rule"], c["fam"], pool[:2 * c["d"]], c["d"], c["L"])
        out["configs"].setdefault("cfg2_batched_%d" % R, {})[names[prec]] = {
            "s": res[0].seconds, "s_per_integral": res[0].seconds / R,
            "points_per_s": R * res[0].points / res[0].seconds, "rel_err_draw0": _rel(res[0], o)}
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
    for label, prec, g in (("fp64", 0, 0.0), ("mixed", 1, 0.0), ("mixed_guard_1e-6", 1, 2.5e-7), ("ff", 2, 0.0)):
        sg.integrate_batch(specs, pool, prec=prec, guard_tol=g)
        res = sg.integrate_batch(specs, pool, prec=prec, guard_tol=g)
        t = res[0].seconds
        errs = [_rel(res[k], o) for k, o in zip(small, refs)]
        out["batch"][label] = {"s": t, "points_per_s": pts / t,
                               "max_rel_err_vs_oracle": max(errs) if errs else None,
                               "oracle_checked_items": len(errs),
                               "max_err_est": max(r.err_est for r in res)}
    # per-class chunk sizes tuned on this subset (sg_autotune_classes), then the
    # guarded batch again with the table
    try:
        ncls = sg.autotune_classes(specs, pool, prec=1, reps=1)
        sg.integrate_batch(specs, pool, prec=1, guard_tol=2.5e-7)
        res = sg.integrate_batch(specs, pool, prec=1, guard_tol=2.5e-7)
        errs = [_rel(res[k], o) for k, o in zip(small, refs)]
        out["batch"]["mixed_guard_1e-6_class_tuned"] = {
            "s": res[0].seconds, "points_per_s": pts / res[0].seconds, "classes": ncls,
            "max_rel_err_vs_oracle": max(errs) if errs else None}
    finally:
        sg.tuning_clear()
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
    # defaults: 20 timed steps after 3 warm-up steps; the 4096-item batch
    # (--workload cfg4, about 200 s per step) one step after one warm-up step
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--per-step", type=int, default=1024, help="integrals per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--prec", default=None, choices=[None, "fp64", "mixed", "ff"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="run the complexity sweep of Section 6 instead of the benchmark")
    ap.add_argument("--sweep-budget", default="4e9", help="largest FP64 evaluation count per run")
    args = ap.parse_args()
    batch = args.workload == "cfg4" and args.impl != "reference"
    if args.steps is None:
        args.steps = 1 if batch else 20
    if args.warmup is None:
        args.warmup = 1 if batch else 3
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cfg4":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
