#!/usr/bin/env python3
"""Benchmark of the LAMP hot path on synthetic workloads shaped like the paper's.

A step is one LAMP iteration (Alg. 2): the fused row sweep, row finalize, fused
column sweep and column finalize over all n x m cost entries, both streams.
The default workload is the high-dimensional one: n = m = 2^15 points in R^64,
x ~ N(0, I), y ~ N(0.5 1, I), uniform marginals, eta = 0, squared Euclidean
cost generated on the fly.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec fp32|bf16_tc]
    python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample

Prints ONE JSON line (rank 0).  value = n*m*K / (device seconds of the K steps),
summed over ranks (each rank solves its own replica: weak scaling, no collective
on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cost-entries/s/iter and time-to-infeasibility≤1e-6 at n=m=2^15 (BF16-TC vs plain FP32)"
UNIT = "cost-entries/s"


def job_throughput(units_per_rank: float, local_seconds: float, dist=None, device=None):
    """Whole-job throughput of weak-scaled replicas: every rank processed
    `units_per_rank` units in its own timed region; the job took the slowest rank's
    time.  Returns (units of all ranks / max seconds, max seconds).  `dist` is
    torch.distributed (any backend) or None for one process."""
    import torch

    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    sec = float(t.item())
    return world * float(units_per_rank) / sec, sec


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the sweeps from one
# ncu capture of this bench's own command line, keyed by (workload, prec, n, d).  A figure is
# reported only while the kernel's sources are those it was taken on (sha256 over the files
# that make up the kernel): after any edit of them the counters no longer describe it and
# `traffic` is null.
NCU_TRAFFIC = {
    ("highdim", "bf16_tc", 32768, 64): {
        "sources": ["paper_2511_11359_gb300/csrc/lamp_tc.cu", "paper_2511_11359_gb300/csrc/lamp_tc.cuh",
                    "paper_2511_11359_gb300/csrc/lamp_async.cuh", "paper_2511_11359_gb300/csrc/lamp_common.cuh"],
        "sha256": "7c3a6dc1c18d6bdc294b81a37c05316fd98c0753effa207139a19e8aa6b02602",
        "row_sweep": 9203712, "col_sweep": 9990144},
    ("image_grid", "fp32", 4096, 0): {
        "sources": ["paper_2511_11359_gb300/csrc/lamp_dense.cu", "paper_2511_11359_gb300/csrc/lamp_async.cuh",
                    "paper_2511_11359_gb300/csrc/lamp_common.cuh"],
        "sha256": "61d2c461514d13861b82ae999b5ce9986d3999b359c1fba50280d88da1925b2a",
        "row_sweep": 67246848 + 244224, "col_sweep": 67254016 + 358912},
}


def sources_digest(sources):
    """sha256 over the concatenated bytes of the given repo files (None if one is missing)."""
    import hashlib

    h = hashlib.sha256()
    for rel in sources:
        try:
            with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), rel), "rb") as f:
                h.update(f.read())
        except OSError:
            return None
    return h.hexdigest()


def ncu_traffic(workload, prec, n, d, which):
    rec = NCU_TRAFFIC.get((workload, prec, n, d))
    if rec is None:
        return None
    return rec[which] if sources_digest(rec["sources"]) == rec["sha256"] else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def make_workload(name: str, rank: int, n=None):
    import workloads as W

    if n is not None:  # reduced sizes, for profiling captures only
        if name == "highdim":
            return W.highdim(n=n, seed=33 + rank)
        if name == "plain_2d":
            return W.plain_2d(n=n, seed=11 + rank)
        if name == "image_grid":
            return W.image_grid(side=int(round(n ** 0.5)), seed=22 + rank)
        if name == "diffloss":
            return W.diffloss(n=n, seed=44 + rank)
        if name == "largescale":
            return W.largescale(n=n, seed=55 + rank)
    if name == "highdim":
        return W.highdim(seed=33 + rank)
    if name == "plain_2d":
        return W.plain_2d(seed=11 + rank)
    if name == "image_grid":
        return W.image_grid(seed=22 + rank)
    if name == "diffloss":
        return W.diffloss(seed=44 + rank)
    if name == "largescale":
        return W.largescale(seed=55 + rank)
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
            return
        # wait (at most 3 s) until nvidia-smi reports, so the timed region is sampled from its
        # start; samples taken before mark() are dropped
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 3.0:
            time.sleep(0.02)

    def mark(self):
        self.first = len(self.lines)

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.first:]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm_, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm_)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(w, max_points: int):
    """A bounded sample of the same workload for the CPU oracle: the first
    max_points sources and targets, marginals renormalised."""
    import oracle as O

    ns = min(w.n, max_points)
    ms = min(w.m, max_points)
    r = w.r[:ns] / w.r[:ns].sum()
    c = w.c[:ms] / w.c[:ms].sum()
    if w.kind == "dense":
        C = np.asarray(w.C[:ns, :ms], dtype=np.float64)
    else:
        C = O.sqeuclid_cost(w.x[:ns], w.y[:ms])
        if w.cost_scale < 0:
            C /= C.max()
        elif w.cost_scale > 0:
            C *= w.cost_scale
    return C, r, c, ns, ms


def time_oracle(w, seconds: float, max_points: int, min_iters: int = 2, fixed_iters: int = 0):
    """Time oracle iterations (Alg. 2, FP64 NumPy) on a bounded sample; returns
    (entries/s/iter, iterations, seconds, sample description)."""
    import oracle as O

    C, r, c, ns, ms = oracle_sample(w, max_points)
    P = O.LampParams(eta=w.eta)
    K, tau1, tau2 = O.resolve_params(C, P)
    ca = O.calpha_of(c, P.alpha)
    st = O.lamp_initial_state(ms)
    st, _ = O.lamp_step(C, r, c, K, tau1, tau2, P.eta, ca, P.beta, st)  # warm-up
    it = 0
    t0 = time.perf_counter()
    while True:
        st, _ = O.lamp_step(C, r, c, K, tau1, tau2, P.eta, ca, P.beta, st)
        it += 1
        el = time.perf_counter() - t0
        if fixed_iters:
            if it >= fixed_iters:
                break
        elif it >= min_iters and el >= seconds:
            break
    el = time.perf_counter() - t0
    desc = (f"{it} Alg. 2 iterations of the FP64 NumPy oracle on the first {ns} x {ms} supports of the "
            f"{w.name} workload (cost matrix precomputed, not timed)")
    return ns * ms * it / el, it, el, desc


GOLDEN_STATES = os.path.join(ROOT, "tests", "golden", "highdim4096_states.npz")


def precision_report(L, torch, devc):
    """Error of the BF16 tensor-core path and of the plain FP32 path against the FP64
    oracle on the unrounded problem, on a 4096 x 4096 sample of the highdim workload
    (the first 4096 source and target points, uniform marginals).  The oracle's states
    come from tests/golden/highdim4096_states.npz (written by the oracle alone): its state
    at the iteration t_stop where its X^t first met infeasibility <= 1e-6, and the
    <C, X> there.  Each GPU path runs as a user would run it (K from its own cost) from
    the Alg. 2 start: to t_stop (errors of nu, theta, log Z, <C, X> at the same t), and
    to its own tolerance (cost at tolerance and iterations)."""
    import oracle as O
    import workloads as W

    z = np.load(GOLDEN_STATES)
    n = int(z["n"])
    w = W.highdim(seed=int(z["seed"]))
    x, y = np.ascontiguousarray(w.x[:n]), np.ascontiguousarray(w.y[:n])
    r = W.uniform_marginal(n)
    c = W.uniform_marginal(n)
    C = O.sqeuclid_cost_expanded(x, y)
    K = float(z["fp32_K"])
    T = int(z["fp32_t_stop"])
    nu_T, th_T, kap_T = z["fp32_nu_stop"], z["fp32_theta_stop"], float(z["fp32_kappa_stop"])
    col_T, logZ_T = O.marginals_from_state(C, r, K, kap_T, nu_T)
    X = r[:, None] * O.dual_to_primal(C, K, kap_T, nu_T)[0]
    cost_T = float((C * X).sum())
    del X
    Cb = O.sqeuclid_cost_expanded(W.bf16_round(x), W.bf16_round(y))
    pert = float(np.abs(Cb - C).max())
    del Cb
    out = {"sample": f"first {n} x {n} supports of the highdim workload, uniform marginals, eta = 0",
           "oracle": {"t_stop": T, "cost_at_t_stop": cost_T, "cost_at_tol": float(z["fp32_cost_stop"]),
                      "K": K},
           "bf16_cost_perturbation_max": pert,
           "bf16_cost_perturbation_note": "max_ij |C(bf16-rounded points) - C|: bounds |OT(C~) - OT(C)|"}
    t_ = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(devc)
    xs, ys, rs, cs = t_(x), t_(y), t_(r), t_(c)
    for prec in ("bf16_tc", "fp32"):
        s = L.Lamp(rs, cs, x=xs, y=ys, cost_scale=1.0, prec=prec, check_every=50)
        s.iterate(T)
        obj = s.objective()
        st = s.get_state()
        lz_err = float((np.abs(st["logZ"] - logZ_T) / (1.0 + np.abs(logZ_T))).max())
        rec = {"at_t_stop": {"nu_max_abs_err": float(np.abs(st["nu"] - nu_T).max()),
                             "theta_max_abs_err": float(np.abs(st["theta"] - th_T).max()),
                             "logZ_max_rel_err": lz_err,
                             "cost_rel_err": abs(obj["cost"] - cost_T) / abs(cost_T),
                             "infeas_gpu": obj["col_res"], "K_gpu": obj["K"]}}
        s.close()
        s = L.Lamp(rs, cs, x=xs, y=ys, cost_scale=1.0, prec=prec, tol=1e-6, check_every=50)
        res = s.solve()
        cat = s.objective()["cost"]
        s.close()
        rec["at_tol"] = {"iters": res["iters"], "oracle_iters": T, "converged": res["converged"],
                         "cost_at_tol": cat,
                         "cost_at_tol_rel_err": abs(cat - float(z["fp32_cost_stop"])) / abs(float(z["fp32_cost_stop"]))}
        out[prec] = rec
    return out


def precision_report_sample(L, torch, devc, w, ns=1024, T=200):
    """Error of the GPU path (float32) against the FP64 oracle on a bounded sample of a
    workload: the first ns source and ns target supports (marginals renormalised; for a
    stored cost the leading ns x ns block), T iterations of Alg. 2 from its start on both
    sides, then the state (nu, theta, log Z) and the objective's quantities (<C, X^t>, the
    column residual, P^eta, the dual bound) compared at the same t.  The oracle solves the
    float64 cost of the float32 inputs; the GPU forms the cost in float32."""
    import oracle as O

    nn, mm = min(w.n, ns), min(w.m, ns)
    r = w.r[:nn] / w.r[:nn].sum()
    c = w.c[:mm] / w.c[:mm].sum()
    t_ = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(devc)
    if w.kind == "dense":
        Cs = np.ascontiguousarray(w.C[:nn, :mm])
        C = Cs.astype(np.float64)
        kw = dict(C=t_(Cs))
    else:
        xs, ys = np.ascontiguousarray(w.x[:nn]), np.ascontiguousarray(w.y[:mm])
        C = O.sqeuclid_cost(xs, ys)
        if w.cost_scale < 0:
            C /= C.max()
        elif w.cost_scale != 1.0:
            C *= w.cost_scale
        kw = dict(x=t_(xs), y=t_(ys), cost_scale=w.cost_scale)
    P = O.LampParams()
    P.eta = w.eta
    K = O.resolve_params(C, P)[0]
    st = O.lamp_run(C, r, c, P, T)
    rep = O.objective_report(C, r, c, K, w.eta, st)
    s = L.Lamp(t_(r), t_(c), eta=w.eta, prec="fp32", check_every=50, **kw)
    s.iterate(T)
    obj = s.objective()
    g = s.get_state()
    s.close()
    rel = lambda a, b: abs(a - b) / max(abs(b), 1e-300)
    return {"sample": f"first {nn} x {mm} supports of the {w.name} workload (marginals renormalised), "
                      f"{T} iterations from the Alg. 2 start, eta = {w.eta}",
            "fp32": {"nu_max_abs_err": float(np.abs(g["nu"] - st.nu).max()),
                     "theta_max_abs_err": float(np.abs(g["theta"] - st.theta).max()),
                     "logZ_max_rel_err": float((np.abs(g["logZ"] - rep["logZ"]) / (1.0 + np.abs(rep["logZ"]))).max()),
                     "cost_rel_err": rel(obj["cost"], rep["cost"]),
                     "col_res_gpu": obj["col_res"], "col_res_oracle": rep["col_res"],
                     "P_eta_rel_err": rel(obj["P_eta"], rep["P_eta"]),
                     "dual_rel_err": rel(obj["dual"], rep["dual"]),
                     "K_gpu": obj["K"], "K_oracle": K}}


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    w = make_workload(args.workload, 0, args.n)
    _, it, el, desc = time_oracle(w, 0, args.cpu_points, fixed_iters=args.warmup)  # warm-up steps
    value, it, el, desc = time_oracle(w, 0, args.cpu_points, fixed_iters=args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / it, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the GPU arm's config keys, with the precision and the sample of this arm
        "config": {"workload": args.workload, "n": w.n, "m": w.m, "d": w.d, "eta": w.eta,
                   "prec": "f64 (NumPy oracle)", "cost": w.kind, "l2": "not applicable (host)",
                   "parallelism": "host, 1 thread",
                   "sample": f"{min(w.n, args.cpu_points)}x{min(w.m, args.cpu_points)}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world):
    import torch
    import paper_2511_11359_gb300 as L

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    devc = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=devc)

    w = make_workload(args.workload, rank, args.n)
    n, m = w.n, w.m
    r = torch.from_numpy(w.r).to(devc)
    c = torch.from_numpy(w.c).to(devc)
    params = dict(eta=w.eta, tol=w.tol, check_every=args.check_every, prec=args.prec)
    if w.kind == "dense":
        C = torch.from_numpy(w.C).to(devc)
        solver = L.Lamp(r, c, C=C, **params)
        h2d_bytes = w.C.nbytes + w.r.nbytes + w.c.nbytes
        flops_per_entry = 0
        bytes_per_entry = 4
    else:
        x = torch.from_numpy(w.x).to(devc)
        y = torch.from_numpy(w.y).to(devc)
        solver = L.Lamp(r, c, x=x, y=y, cost_scale=w.cost_scale, **params)
        h2d_bytes = w.x.nbytes + w.y.nbytes + w.r.nbytes + w.c.nbytes
        flops_per_entry = 2 * w.d
        bytes_per_entry = 0
    stream = torch.cuda.current_stream()
    launches = solver.launches_per_iteration()

    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=devc)

    for _ in range(args.warmup):
        solver.iterate(1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # clocks are sampled over every GPU-timed measurement of the line: the timed steps, the
    # per-kernel timing, the end-to-end steps, the float32 comparison and the solves to tolerance
    sampler = ClockSampler(local)
    sampler.start()
    sampler.mark()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        solver.iterate(1)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    # per-kernel device times, measured with events between the launches
    kern_ms = solver.time_kernels(max(3, min(args.steps, 10)))
    value, total_s = job_throughput(n * m * args.steps, total_ms / 1e3, dist, devc)
    total_ms = total_s * 1e3

    # end to end through the C ABI with host buffers: every step uploads the inputs
    # from pinned host memory, runs one iteration and reads back nu and the residual
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        if w.kind == "dense":
            hst = L.LampHost(w.r, w.c, C=w.C, **params)
            a_h, b_h = pin(w.C), None
        else:
            hst = L.LampHost(w.r, w.c, x=w.x, y=w.y, cost_scale=w.cost_scale, **params)
            a_h, b_h = pin(w.x), pin(w.y)
        r_h, c_h = pin(w.r), pin(w.c)
        nu_h = torch.empty(m, dtype=torch.float64).pin_memory().numpy()
        for _ in range(2):
            hst.step(1, a_h, b_h, r_h, c_h, nu_out=nu_h)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            hst.step(1, a_h, b_h, r_h, c_h, nu_out=nu_h)
        el = time.perf_counter() - t0
        hst.close()
        e2e_value, _ = job_throughput(n * m * args.e2e_steps, el, dist, devc)
        # the copies alone: the same pinned host buffers to device tensors, CUDA events
        srcs = [a for a in (a_h, b_h, r_h, c_h) if a is not None]
        dsts = [torch.empty(a.shape, dtype=torch.from_numpy(a).dtype, device=devc) for a in srcs]
        cms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for dd, a in zip(dsts, srcs):
                dd.copy_(torch.from_numpy(a), non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            cms.append(e0.elapsed_time(e1))
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d_bytes),
               "d2h_bytes_per_step": int(8 + 8 * m), "steps": args.e2e_steps,
               "ms_per_step": 1e3 * el / args.e2e_steps, "h2d_copy_ms": min(cms)}

    info = {}
    if rank == 0 and args.prec == "bf16_tc" and w.kind != "dense" and not args.no_fp32_compare:
        # the plain float32 path on the same problem, same timing protocol
        s32 = L.Lamp(r, c, x=x, y=y, cost_scale=w.cost_scale, **dict(params, prec="fp32"))
        for _ in range(args.warmup):
            s32.iterate(1)
        torch.cuda.synchronize()
        ev32 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.fp32_steps)]
        for i in range(args.fp32_steps):
            flush.zero_()
            ev32[i][0].record(stream)
            s32.iterate(1)
            ev32[i][1].record(stream)
        torch.cuda.synchronize()
        ms32 = sum(a.elapsed_time(b) for a, b in ev32) / args.fp32_steps
        k32 = s32.time_kernels(3)
        fp32 = {"value": n * m / (ms32 / 1e3), "ms_per_step": ms32, "kernel_ms": k32}
        if args.ttt:
            torch.cuda.synchronize()
            t0 = time.perf_counter()  # from context creation: the K pass and the prime pass count
            s32b = L.Lamp(r, c, x=x, y=y, cost_scale=w.cost_scale, max_iter=args.ttt_max_iter,
                          **dict(params, prec="fp32"))
            rr = s32b.solve()
            fp32["time_to_tol"] = {"seconds": time.perf_counter() - t0, "iters": rr["iters"],
                                   "infeas": rr["infeas"], "converged": rr["converged"], "tol": w.tol}
            fp32["cost_at_tol"] = s32b.objective()["cost"]
            s32b.close()
        s32.close()
        info["fp32_path"] = fp32
    if rank == 0 and args.ttt:
        # time to infeasibility <= tol from the Alg. 2 start: context creation (K pass,
        # row-shift prime pass) and lamp_solve
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = L.Lamp(r, c, x=x, y=y, cost_scale=w.cost_scale, max_iter=args.ttt_max_iter,
                    **params) if w.kind != "dense" else L.Lamp(r, c, C=C, max_iter=args.ttt_max_iter, **params)
        res = s2.solve()
        el = time.perf_counter() - t0
        info["time_to_tol"] = {"seconds": el, "iters": res["iters"], "infeas": res["infeas"],
                               "converged": res["converged"], "tol": w.tol}
        info["cost_at_tol"] = s2.objective()["cost"]
        s2_state = s2.get_state()
        s2.close()
        if w.eta > 0:
            # for eta > 0 the rule above also waits for 1 - kappa_t eta <= tol; the same solve
            # stopped by the infeasibility alone (lamp_params.infeas_only)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p3 = dict(params, infeas_only=1)
            s3 = L.Lamp(r, c, x=x, y=y, cost_scale=w.cost_scale, max_iter=args.ttt_max_iter,
                        **p3) if w.kind != "dense" else L.Lamp(r, c, C=C, max_iter=args.ttt_max_iter, **p3)
            r3 = s3.solve()
            info["time_to_tol_infeas_only"] = {"seconds": time.perf_counter() - t0, "iters": r3["iters"],
                                               "infeas": r3["infeas"], "converged": r3["converged"],
                                               "tol": w.tol, "cost": s3.objective()["cost"]}
            s3.close()
        if w.kind != "dense":
            # the autograd form: lamp_ot_loss forward (context creation, solve to tol, objective)
            # and the hand-written backward (lamp_grad)
            xg = x.clone().requires_grad_(True)
            yg = y.clone().requires_grad_(True)
            # PyTorch starts its autograd device threads on the first backward of a process
            # (0.1 - 1.5 s on the Arm hosts): a tiny unrelated backward takes that cost
            warm = torch.ones(2, device=devc, requires_grad=True)
            (warm * 2.0).sum().backward()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = L.lamp_ot_loss(xg, yg, r=r, c=c, eta=w.eta, cost_scale=w.cost_scale, prec=args.prec, tol=w.tol,
                                  max_iter=args.ttt_max_iter, check_every=args.check_every)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            loss.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            info["autograd_form"] = {"forward_s": t1 - t0, "backward_s": t2 - t1, "total_s": t2 - t0,
                                     "loss": float(loss.item()),
                                     "grad_finite": bool(torch.isfinite(xg.grad).all() and torch.isfinite(yg.grad).all())}
            # lamp_grad alone on the converged context of the timed solve (s2 was closed: a fresh
            # context on its final state), first call (allocates its buffers) and a repeat
            sg = L.Lamp(r, c, x=x, y=y, cost_scale=w.cost_scale, **params)
            st2 = s2_state
            sg.set_state(st2["nu"], st2["theta"], st2["kappa"], st2["t"], st2["row_shifts"])
            gms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                sg.grad()
                e1.record(stream)
                torch.cuda.synchronize()
                gms.append(e0.elapsed_time(e1))
            sg.close()
            info["autograd_form"]["lamp_grad_ms"] = {"first_call": gms[0], "repeat": min(gms[1:]),
                                                     "includes": "one evaluation pass + one pass per side"}

    clocks = sampler.stop()
    if rank == 0 and args.workload == "highdim" and not args.no_precision and w.n == 1 << 15:
        info["precision_vs_fp64_oracle"] = precision_report(L, torch, devc)
    elif rank == 0 and args.workload != "highdim" and not args.no_precision:
        info["precision_vs_fp64_oracle"] = precision_report_sample(L, torch, devc, w)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, src = load_peaks()
    dom = 0 if kern_ms[0] >= kern_ms[2] else 2
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if bytes_per_entry:
        achieved = n * m * bytes_per_entry / (kern_ms[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": ncu_traffic(args.workload, args.prec, n, w.d, "row_sweep" if dom == 0 else "col_sweep"),
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "what": "stored C bytes of the " + ("row" if dom == 0 else "column") + " sweep"}
    elif args.prec == "bf16_tc" or w.d <= 8:
        # tensor-core sweeps, and the packed f32x2 direct-form sweeps (d <= 8): two ex2 per entry
        rate = L.measure_ex2_rate()
        peak = sms * rate * mhz * 1e6 / 1e12
        achieved = n * m * 2 / (kern_ms[dom] / 1e3) / 1e12
        form = "tcgen05 x.y" if args.prec == "bf16_tc" else "f32x2 direct |x - y|^2"
        mufu = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tex2/s", "frac": achieved / peak,
                "what": "MUFU ex2 of the " + ("row" if dom == 0 else "column") + f" sweep ({form}; 2 ex2 per entry: "
                        "streams A, B)",
                "peak_source": f"{sms} SMs x {rate:.2f} ex2/clk/SM (measured, lamp_measure_ex2_rate) x {mhz:.0f} MHz"}
        if args.prec == "bf16_tc":
            # MUFU binds: 16 entries / clk / SM, against ~21 for the FP32 pipe at 6 lane-ops per entry
            roof = dict(mufu)
        else:
            # the FP32 pipe binds the direct form: float32 lane operations per entry of a regular
            # iteration: d sub + d mul/fma (cost); stream A add + 2 fma (compensated exponent) +
            # fma (weighted sum); stream B, through the shared row shift, add + fma + fma; at d = 3
            # that is 13 lane-ops, 9.8 entries / clk / SM, against 16 for MUFU
            lanes = 2 * w.d + 7
            fpeak = sms * 128 * mhz * 1e6 / 1e12
            fach = n * m * lanes / (kern_ms[dom] / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": fach, "peak": fpeak, "unit": "Tlane-op/s", "frac": fach / fpeak,
                    "what": "FP32-pipe lane operations of the " + ("row" if dom == 0 else "column") +
                            f" sweep ({form}; {lanes} lane-ops per entry)",
                    "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz", "mufu": mufu}
        roof["traffic"] = ncu_traffic(args.workload, args.prec, n, w.d, "row_sweep" if dom == 0 else "col_sweep")
        roof["traffic_unit"] = "bytes per launch (ncu dram read + write)"
    else:
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flop x max SM clock
        achieved = n * m * flops_per_entry / (kern_ms[dom] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "what": "fp32 x.y FMA of the " + ("row" if dom == 0 else "column") + " sweep",
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"}
    roof["kernel_ms"] = {"row_sweep": kern_ms[0], "row_fin": kern_ms[1], "col_sweep": kern_ms[2],
                         "col_fin": kern_ms[3]}
    roof["peak_of"] = src
    if not bytes_per_entry and (args.prec == "bf16_tc" or w.d <= 8):
        # the whole iteration against the MUFU rate, counting 2 ex2 per entry per iteration
        # (one per marginal evaluation of Alg. 2, Step 1) and, as built, 4: with O(n + m)
        # memory each of the two evaluations needs its row normalisers before its column
        # sums, so every entry is formed once in the row sweep and once in the column sweep
        it_s = (total_ms / args.steps) / 1e3
        roof["iteration"] = {
            "ms": total_ms / args.steps, "peak_Tex2_s": mufu["peak"],
            "frac_2ex2_per_entry": n * m * 2 / it_s / 1e12 / mufu["peak"],
            "frac_4ex2_per_entry_as_built": n * m * 4 / it_s / 1e12 / mufu["peak"]}

    cpu = None
    if not args.no_cpu_baseline:
        v, it, el, desc = time_oracle(w, args.cpu_seconds, args.cpu_points)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "bf16 x.y, f32 accumulate and exp",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "m": m, "d": w.d, "eta": w.eta, "prec": args.prec,
                   "cost": w.kind, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas{world}"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    line.update(info)
    print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


# the paper's Table 1: row-LSE reduction latency (ms) of its fused + warp-tiled kernel on an
# RTX 4090 (one stream, precision not stated), for context only
PAPER_TABLE1_FUSED_WT_MS = {1024: 0.12, 4096: 1.30, 16384: 17.13, 65536: 252.5}


def run_lse_table(args):
    """Row sweep (G1: row sums of both streams, i.e. two row LSEs) at the n of the paper's
    Table 1, for a stored n x n float32 C ~ U[0,1) and for on-the-fly |x - y|^2 with
    x, y ~ U[0,1]^3; mean CUDA-event time of the row-sweep launch over `steps` iterations."""
    import torch
    import paper_2511_11359_gb300 as L

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rows = []
    for n in sorted(PAPER_TABLE1_FUSED_WT_MS):
        g = torch.Generator(device=dev).manual_seed(1000 + n)
        r = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
        entry = {"n": n, "paper_fused_wt_ms_rtx4090_one_stream": PAPER_TABLE1_FUSED_WT_MS[n]}
        C = torch.rand((n, n), generator=g, device=dev, dtype=torch.float32)
        s = L.Lamp(r, r, C=C, K=1.0)
        s.iterate(args.warmup)
        entry["stored_C_row_sweep_ms"] = s.time_kernels(args.steps)[0]
        s.close()
        del C
        torch.cuda.empty_cache()
        x = torch.rand((n, 3), generator=g, device=dev, dtype=torch.float32)
        y = torch.rand((n, 3), generator=g, device=dev, dtype=torch.float32)
        s = L.Lamp(r, r, x=x, y=y, K=3.0)
        s.iterate(args.warmup)
        entry["points_d3_row_sweep_ms"] = s.time_kernels(args.steps)[0]
        s.close()
        entry["stored_C_entries_per_s"] = n * n / (entry["stored_C_row_sweep_ms"] / 1e3)
        entry["points_d3_entries_per_s"] = n * n / (entry["points_d3_row_sweep_ms"] / 1e3)
        rows.append(entry)
    print(json.dumps({"metric": "row-LSE sweep time at the shapes of the paper's Table 1 (two streams per sweep)",
                      "unit": "ms", "higher_is_better": False, "data": "synthetic", "steps": args.steps,
                      "warmup": args.warmup, "lse_table": rows}), flush=True)


def run_grad_only(args):
    """lamp_grad alone on the workload (tensor cores for d > 8): `warmup` iterations of Alg. 2,
    then `steps` calls of lamp_grad on that state, each timed with CUDA events (the first call
    also runs the evaluation pass and allocates the pass's buffers; later calls reuse both)."""
    import torch
    import paper_2511_11359_gb300 as L

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = make_workload(args.workload, 0, args.n)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    s = L.Lamp(t(w.r), t(w.c), x=t(w.x), y=t(w.y), cost_scale=w.cost_scale, eta=w.eta, prec=args.prec,
               check_every=args.check_every)
    s.iterate(args.warmup)
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.grad()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    s.close()
    print(json.dumps({"metric": "lamp_grad time (envelope gradient, both sides)", "unit": "ms",
                      "higher_is_better": False, "workload": args.workload, "n": w.n, "m": w.m, "d": w.d,
                      "prec": args.prec, "first_call_ms": ms[0],
                      "repeat_ms": min(ms[1:]) if len(ms) > 1 else None, "calls": len(ms)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="highdim")
    ap.add_argument("--n", type=int, default=None, help="override n = m (profiling captures only)")
    ap.add_argument("--prec", default=None, choices=["fp32", "bf16_tc"],
                    help="default: bf16_tc for point clouds with d > 8, fp32 otherwise")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=5)
    ap.add_argument("--check-every", type=int, default=50)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-infeasibility measurement")
    ap.add_argument("--ttt-max-iter", type=int, default=200000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the error report of both GPU precisions against the FP64 oracle (highdim)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-points", type=int, default=2048)
    ap.add_argument("--grad-only", action="store_true",
                    help="time lamp_grad alone (after --warmup iterations, --steps calls) instead of the bench")
    ap.add_argument("--lse-table", action="store_true",
                    help="row-sweep timings at the paper's Table 1 sizes (n = 1024 .. 65536) instead of the bench")
    args = ap.parse_args()
    args.ttt = not args.no_ttt
    if args.prec is None:
        args.prec = "bf16_tc" if args.workload == "highdim" else "fp32"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.warmup < 3 and args.impl == "gpu":
        raise SystemExit("--warmup must be >= 3")
    if args.lse_table:
        run_lse_table(args)
    elif args.grad_only:
        run_grad_only(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
