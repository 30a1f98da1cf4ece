#!/usr/bin/env python
"""Throughput of the tensor butterfly apply u = K f (Alg. 2) on GB300.

One step = one full apply (source leaves, source transfers, mid-level core,
target transfers, target leaves) of the workload's operator to its batch of
right-hand sides, inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU (torchrun): each rank holds its own copy of the operator and applies
its own batch of right-hand sides (replicas, weak scaling); the timed region
is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import ctypes
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

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "TB apply Gpts·RHS/s & % roofline, mixed/batched vs FP64 plain at stated rel err"
UNIT = "Gpts*RHS/s"
DEFAULT_WORKLOAD = "helmholtz3d_n256"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(W.WORKLOADS))
    p.add_argument("--precision", type=int, default=None, help="0 c128, 1 c64, 2 split-bf16")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    p.add_argument("--err-samples", type=int, default=4096,
                   help="sampled outputs of the error check (the stored oracle values of the full-size "
                        "3-D Helmholtz configuration when they apply; else the live oracle, capped)")
    p.add_argument("--profile-only", action="store_true", help="eager applies only (for ncu)")
    p.add_argument("--n", type=int, default=None, help="points per axis of a reduced-size copy (profiling)")
    p.add_argument("--nv", type=int, default=None, help="right-hand sides of a reduced-size copy (profiling)")
    p.add_argument("--level-schedule", type=int, default=0,
                   help="non-separable handles: tb_options.level_schedule (0 rule, 1 per-mode, 2 fused)")
    p.add_argument("--core-mode", type=int, default=0,
                   help="tb_options.core_mode (0 rule, 1 stored cores, 2 regenerated in the one-RHS forward core)")
    p.add_argument("--mode-slices", type=int, default=0,
                   help="tb_options.mode_slices (0 rule / tuner; 1, 2, 4 thread groups per column of a mode launch)")
    p.add_argument("--sep-schedule", type=int, default=0,
                   help="separable handles: tb_options.sep_schedule (0 rule; the tuner may replace it)")
    return p.parse_args()


def workload(args):
    w = W.WORKLOADS[args.workload]
    if not args.n and not args.nv:
        return w
    n = args.n or w.n
    kw = {}
    if w.kind == W.HELMHOLTZ and n != w.n:   # keep the points per wavelength of the full workload
        kw["params"] = (w.params[0] * n / w.n,)
    return W.small(args.workload, n, nv=args.nv or w.nv, **kw)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by workload,
# precision and pass; see profiles/ for the command.  Entries are removed when
# the kernel changes.
TRAFFIC = {}
# k_core_tc, one launch of helmholtz3d_n256 (16 RHS): ncu dram__bytes_read.sum + dram__bytes_write.sum
TRAFFIC[("helmholtz3d_n256", 2, "core@l2")] = 6.00e9 + 0.21187e9
# every per-mode register pass of fourier6d_n16 reads and writes the whole tensor once
TRAFFIC.update({("fourier6d_n16", 1, f"sep_reg@l{k}"): 1.073863e9 + 1.025651e9 for k in range(6)})


def permode_order(d, m, o, first0=False, last_d1=False):
    """The per-mode launch order of a pass (the library's rule): fewest complex
    multiply-adds, mode 0 first for LeafIn / Split, mode d-1 last for Gather."""
    import itertools
    best, best_f = None, None
    for p in itertools.permutations(range(d)):
        if (first0 and p[0] != 0) or (last_d1 and p[-1] != d - 1):
            continue
        cur, f = list(m), 0
        for k in p:
            t = m[k] * o[k]
            for j in range(d):
                if j != k:
                    t *= cur[j]
            f += t
            cur[k] = o[k]
        if best_f is None or f <= best_f:   # ties: the last order, as the library
            best, best_f = p, f
    return best


def level_mode_bytes(info, w, nv, es):
    """Bytes each level pass streams as d mode-product launches: every launch
    reads its input and writes its output once (level tensors, the user tensor
    and the mode intermediates), factors excluded; each pass in its launch order."""
    d, Lc = info["d"], info["Lc"]
    P = 2 ** (2 * d * Lc)
    cb = [w.n >> info["L"]] * d
    out = {}

    def chain(m, o, in_total, out_total, **rule):
        b = in_total
        cur = list(m)
        for k in permode_order(d, m, o, **rule)[:-1]:
            cur[k] = o[k]
            b += 2 * P * nv * es * math.prod(cur)
        return b + out_total

    N = w.N
    user = N * nv * es
    rs, rt = info["rank_src"], info["rank_tgt"]
    tile = lambda R: P * nv * es * math.prod(R)
    out["leaf_in@l0"] = chain(cb, rs[0], user, tile(rs[0]), first0=True)
    out["leaf_out@l0"] = chain(rt[0], cb, tile(rt[0]), user)
    for l in range(1, Lc + 1):
        out[f"split@l{l}"] = chain([2 * r for r in rs[l - 1]], rs[l], tile(rs[l - 1]), tile(rs[l]), first0=True)
        out[f"gather@l{l}"] = chain(rt[l], [2 * r for r in rt[l - 1]], tile(rt[l]), tile(rt[l - 1]), last_d1=True)
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            j = json.load(fh)
        return {"hbm_gbs": j["hbm_gbs"], "bf16_tflops": j["bf16_tflops"],
                "bf16_tflops_sustained": j.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def cpu_baseline(w, f_np, budget_s=15.0, seed=4096):
    """The oracle direct sum, as it stands, on a bounded sample of output points."""
    import oracle
    oracle.build()
    xs, ys = W.grids(w)
    probe = W.sample_targets(w, 2, seed=seed + 1)
    t0 = time.perf_counter()
    oracle.apply(w.kind, w.params, xs, ys, f_np, probe)
    per = max((time.perf_counter() - t0) / 2, 1e-6)
    # the direct sum parallelizes over targets: keep at least one target per thread
    count = int(max(oracle.threads(), min(4096, budget_s / per * oracle.threads())))
    rows = W.sample_targets(w, count, seed=seed)
    t0 = time.perf_counter()
    oracle.apply(w.kind, w.params, xs, ys, f_np, rows)
    t = time.perf_counter() - t0
    nv = f_np.shape[-1]
    return {"value": count * nv / t / 1e9, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{count} sampled output points x {nv} RHS of the direct FP64 sum ({t:.1f} s)"}


def reference_arm(args, ws, rank):
    w = workload(args)
    if rank != 0:
        return
    import oracle
    oracle.build()
    f = W.rhs(w).numpy()
    xs, ys = W.grids(w)
    probe = W.sample_targets(w, 2, seed=7)
    t0 = time.perf_counter()
    oracle.apply(w.kind, w.params, xs, ys, f, probe)
    per = max((time.perf_counter() - t0) / 2, 1e-6)
    total = max(args.steps + args.warmup, 1)
    count = int(max(oracle.threads(), min(4096, 120.0 / total / per * oracle.threads())))
    times = []
    for s in range(args.warmup + args.steps):
        rows = W.sample_targets(w, count, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.apply(w.kind, w.params, xs, ys, f, rows)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = count * w.nv / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "d": w.d, "nv": w.nv, "tol": w.tol},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{count} sampled output points x {w.nv} RHS per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


GOLDEN = os.path.join(ROOT, "tests", "golden")
# direct-sum work the live error check may spend (kernel evaluations)
LIVE_ORACLE_EVALS = 2.0e9


def sampled_reference(w, f_np, count):
    """Oracle values on sampled outputs: (rows, u_ref, cols, v_ref, source).

    For the full-size 3-D Helmholtz configuration the values stored in
    tests/golden/helmholtz3d_n256.npz (written by the script beside it, which
    calls only oracle/) are used when the seeded inputs reproduce their
    fingerprint; otherwise the direct sum runs here on `count` outputs, capped so
    that it stays within a bounded number of kernel evaluations."""
    path = os.path.join(GOLDEN, f"{w.name}.npz")
    if os.path.exists(path):
        z = np.load(path)
        rows = z["rows"]
        if np.array_equal(f_np.reshape(-1, w.nv)[rows[:16]], z["fingerprint"]):
            k = min(count, len(rows))
            return rows[:k], z["u"][:k], z["cols"][:k], z["v"][:k], "stored oracle values"
    import oracle
    count = int(max(16, min(count, LIVE_ORACLE_EVALS / w.N)))
    rows = W.sample_targets(w, count, seed=4096)
    cols = W.sample_targets(w, count, seed=4097)
    return (rows, oracle.workload_apply(w, f_np, rows), cols, oracle.workload_apply_adjoint(w, f_np, cols),
            "live oracle")


def rel_err_rows(x_dev, nv, rows, ref):
    x = x_dev.reshape(-1, nv)[torch.from_numpy(np.asarray(rows)).to(x_dev.device)].cpu().to(torch.complex128).numpy()
    per = np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref)), float(per.max())


def step_bytes(info, w, nv, prec):
    """Algorithmic bytes of one apply: input and output tensors, factors and
    cores at their stored sizes, and the one mid-level exchange,
    bd nv (N_in + N_out) + bf (V, W, U, P entries) + bf (core entries)
    + 2 bd nv min(|F_mid|, |G_mid|)."""
    bd = 16 if prec == 0 else 8
    bf = bd
    mid = min(info["mid_src_entries"], info["mid_tgt_entries"])
    return bd * nv * 2 * w.N + bf * info["factor_entries"] + bf * info["core_entries"] + 2 * bd * nv * mid


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return
    torch.cuda.set_device(local)
    import paper_2411_03029_gb300 as tb
    tb.build.build()
    w = workload(args)
    prec = args.precision if args.precision is not None else w.precision
    mask = (1 << prec) | ((1 << tb.PREC_C128) if not args.no_fp64 else 0)
    op = tb.from_workload(w, precisions=mask, use_graphs=not args.profile_only, precision=prec,
                          sep_schedule=args.sep_schedule, level_schedule=args.level_schedule,
                          core_mode=args.core_mode, mode_slices=args.mode_slices)
    info = op.info()
    nv = w.nv
    tune_s = None
    if not args.no_autotune:                # launch shapes for this nv and precision (tb_autotune)
        t0 = time.perf_counter()
        op.autotune(nv, prec)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
    f_host = W.rhs(w)                       # complex128, CPU
    if ws > 1:                              # each replica applies its own batch
        f_host = W.complex_gaussian(f_host.shape, 10_000 + rank)
    dt = tb.dtype_of(prec)
    f = f_host.to(dt).cuda()
    u = torch.empty_like(f)
    stream = torch.cuda.Stream()
    N = w.N

    if args.profile_only:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup + args.steps):
                op.apply(f, prec, out=u)
        stream.synchronize()
        # sizes for scaling counter captures of this (possibly reduced) copy to the full workload
        core_bytes = 8 * info["core_entries"] + 8 * nv * (info["mid_src_entries"] + info["mid_tgt_entries"])
        print(json.dumps({"profile_only": True, "workload": w.name, "n": w.n, "nv": nv,
                          "core_entries": info["core_entries"], "mid_src_entries": info["mid_src_entries"],
                          "mid_tgt_entries": info["mid_tgt_entries"], "core_pass_bytes_c64": core_bytes,
                          "ranks_src": info["rank_src"], "ranks_tgt": info["rank_tgt"]}))
        return

    # ---------------------------------------------------- timed region (graph replay)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            op.apply(f, prec, out=u)
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                op.apply(f, prec, out=u)
            ev1.record(stream)
        stream.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        # the same K steps launched eagerly (legacy stream: no graph) with CUDA
        # events recorded around every pass on that stream (roofline)
        op.profile(True)
        for _ in range(args.steps):
            tb._check(tb.lib().tb_apply(op._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                        nv, prec, ctypes.c_void_p(0)))
        torch.cuda.synchronize()
        op.profile(False)
    stats = op.profile_stats()
    ms = max_over_ranks(ws, ms)
    # the adjoint apply K^H on the same batch (graph replay, same step count)
    v = torch.empty_like(f)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            op.apply_adjoint(f, prec, out=v)
    stream.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            op.apply_adjoint(f, prec, out=v)
        ev1.record(stream)
    stream.synchronize()
    ms_adj = max_over_ranks(ws, ev0.elapsed_time(ev1) / args.steps)
    adjoint = {"value": ws * N * nv / (ms_adj * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_adj}
    value = ws * N * nv / (ms * 1e-3) / 1e9
    # kernel launches of one apply, counted from the per-pass event records
    launches_per_step = int(round(sum(s["kernels"] for s in stats) / max(args.steps, 1))) if stats else 0

    pk = peaks()
    # the dominant kernel: the pass whose single launch takes longest (a level
    # pass is d mode-product launches, the core one launch per 16 RHS)
    dom = max(stats, key=lambda s: s["ms_total"] / max(s["kernels"], 1)) if stats else None
    roof = None
    if dom:
        per_launch_ms = dom["ms_total"] / dom["kernels"]
        per_pass = dom["kernels"] / dom["launches"]
        bytes_launch = dom["bytes"] / per_pass
        flops_launch = dom["flops"] / per_pass
        achieved_gbs = bytes_launch / (per_launch_ms * 1e-3) / 1e9
        name = f'{dom["name"]}@l{dom["level"]}'
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved_gbs,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved_gbs / pk["hbm_gbs"],
                "peak_source": pk["source"], "traffic": TRAFFIC.get((w.name, prec, name)),
                "bytes_per_launch": bytes_launch, "flops_per_launch": flops_launch, "ms_per_launch": per_launch_ms,
                "tflops": flops_launch / (per_launch_ms * 1e-3) / 1e12,
                "flop_per_byte": flops_launch / max(bytes_launch, 1),
                "share_of_step": dom["ms_total"] / max(sum(s["ms_total"] for s in stats), 1e-9)}
    if roof is not None:
        b_step = step_bytes(info, w, nv, prec)
        roof["step_bytes"] = b_step
        roof["step_achieved"] = b_step / (ms * 1e-3) / 1e9
        roof["step_frac"] = roof["step_achieved"] / pk["hbm_gbs"]
    try:
        fp32_peak = tb.alu_peak(tb.PREC_C64)
        fp64_peak = tb.alu_peak(tb.PREC_C128)
    except Exception:
        fp32_peak = fp64_peak = None
    passes = [{"pass": f'{s["name"]}@l{s["level"]}', "ms": s["ms_total"] / s["launches"],
               "kernels": s["kernels"] // max(s["launches"], 1),
               "GBps": s["bytes"] / (s["ms_total"] / s["launches"] * 1e-3) / 1e9,
               "TFLOPs": s["flops"] / (s["ms_total"] / s["launches"] * 1e-3) / 1e12} for s in stats]
    alu = fp64_peak if prec == tb.PREC_C128 else fp32_peak
    for p_ in passes:
        p_["hbm_frac"] = p_["GBps"] / pk["hbm_gbs"]
        # CUDA-core passes against the measured FMA peak (the split-BF16 core runs on the tensor cores)
        if alu and (not p_["pass"].startswith("core") or prec != tb.PREC_C64_SPLITBF16):
            p_["alu_frac"] = p_["TFLOPs"] / alu
    mode_traffic = level_mode_bytes(info, w, nv, 8 if prec != tb.PREC_C128 else 16)
    for p_ in passes:
        if p_["pass"] in mode_traffic:   # bytes the per-mode launches stream, intermediates included
            p_["mode_bytes"] = mode_traffic[p_["pass"]]
            p_["mode_GBps"] = mode_traffic[p_["pass"]] / (p_["ms"] * 1e-3) / 1e9

    # --------------------------------------------------- end to end with host buffers
    f_pin = f_host.to(dt).pin_memory().numpy()
    u_pin = torch.empty(f_pin.shape, dtype=dt).pin_memory().numpy()

    # every step copies its input from pinned host memory and its result back;
    # tb_apply_host_batch overlaps step i's apply with the copies of steps i + 1 and i - 1
    e2e_steps = max(1, min(args.steps, 10))
    op.apply_host_batch([f_pin] * 2, [u_pin] * 2, prec)   # warm-up: pipeline buffers and graphs
    barrier(ws)
    t0 = time.perf_counter()
    op.apply_host_batch([f_pin] * e2e_steps, [u_pin] * e2e_steps, prec)
    t_e2e = max_over_ranks(ws, (time.perf_counter() - t0) / e2e_steps)
    es = 16 if prec == tb.PREC_C128 else 8
    e2e = {"value": ws * N * nv / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": N * nv * es,
           "d2h_bytes_per_step": N * nv * es, "ms_per_step": t_e2e * 1e3, "steps": e2e_steps,
           "api": "tb_apply_host_batch"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {0: "c128", 1: "c64", 2: "c64+bf16x2"}[prec], "data": "synthetic",
           "config": {"workload": w.name, "kernel": w.description, "d": w.d, "n": w.n, "nv": nv, "tol": w.tol,
                      "L": info["L"], "ranks_src": info["rank_src"], "ranks_tgt": info["rank_tgt"],
                      "rank_min": info["rank_min"], "rank_max": info["rank_max"],
                      "core_entries": info["core_entries"], "build_s": info["build_seconds"],
                      "l2": "inputs larger than L2 (no flush)", "graph": True,
                      "autotune_s": tune_s},
           "roofline": roof, "passes": passes, "adjoint": adjoint, "e2e": e2e,
           "alu_peak": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak, "kind": "measured",
                        "how": "tb_alu_peak: independent FMA chains on every SM, CUDA-event timed"},
           "gpu_launches": launches_per_step * args.steps}

    if rank == 0:
        f_np = f_host.numpy()
        refs = None
        if args.err_samples > 0:
            refs = sampled_reference(w, f_np, args.err_samples)
            rows, u_ref, cols, v_ref, src = refs
            e_all, e_max = rel_err_rows(u, nv, rows, u_ref)
            ea_all, ea_max = rel_err_rows(v, nv, cols, v_ref)
            out["rel_err_sampled"] = e_all
            out["rel_err_sampled_max_rhs"] = e_max
            out["rel_err_adjoint_sampled"] = ea_all
            out["rel_err_adjoint_max_rhs"] = ea_max
            out["rel_err_samples"] = {"outputs": int(len(rows)), "rhs": nv, "reference": src}
            out["rel_err_bound"] = w.bound
        if not args.no_fp64 and prec != tb.PREC_C128:
            f64 = f_host.cuda()
            u64 = torch.empty_like(f64)
            with torch.cuda.stream(stream):
                op.apply(f64, tb.PREC_C128, out=u64)
                stream.synchronize()
                k64 = max(1, min(3, args.steps))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(k64):
                    op.apply(f64, tb.PREC_C128, out=u64)
                e1.record(stream)
            stream.synchronize()
            ms64 = e0.elapsed_time(e1) / k64
            out["fp64_plain"] = {"value": N * nv / (ms64 * 1e-3) / 1e9, "ms_per_step": ms64,
                                 "rel_err_sampled": rel_err_rows(u64, nv, refs[0], refs[1])[0]
                                 if refs is not None else None}
            del f64, u64
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, f_np)
    out["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(out), flush=True)
    op.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
