"""Benchmark: block-coordinate Frank-Wolfe solves of semi-relaxed OT on GB300.

Default (the headline): one step = one complete solve of colour4096_fp32
(m = n = 4096 RGB-like points from seeded 8-component Gaussian mixtures,
Dirichlet(1) target weights, rho = 10, squared-Euclidean cost on the fly)
to relative duality gap 1e-6 with pairwise steps and the exact line search,
the certificate (Thm 2) taken every epoch. `value` = block updates per
second over the timed solves; `ms_per_step` = time to gap. Inputs are
resident in HBM when the timed region starts; L2 is flushed (256 MB write)
between timed steps.

Other workloads (--workload):
  colour256_fp64       FP64 BCFW, decay rule, cyclic, 200 epochs
  colour_batch512      512 instances, m, n ~ U{64..2048}, one persistent launch
  feature8192_d128     BF16 tensor-core cost (d = 128) + FP32 solve to 1e-6
  colour_batch64_2048  64 x (2048 x 2048): batched solve + adjoint (backward); the
                       colour-transfer pass over the same plans is timed on its own

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun with N > 1: single-instance workloads run one replica per
rank (weak scaling); batched workloads split the instances over the ranks
by longest-processing-time-first on m*n (strong scaling). No data-path
collective either way; value = all ranks' block updates / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "block-updates/s"
VARIANTS = {"BCFW": 0, "BCAFW": 1, "BCPFW": 2}
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (Blackwell)
FLOPS_PER_GRAD = 8        # d = 3 cost (3 sub, 3 mul/fma) + residual add + compare
BATCH_WORKLOADS = ("colour_batch512", "colour_batch64_2048")

# DRAM bytes (read + write) per launch of a workload's dominant kernel from one
# ncu capture (summaries in profiles/), valid only while the sources that kernel
# is built from are the ones captured: their digest at capture time must match.
CAPTURED_TRAFFIC = {
    ("colour4096_fp32", "roofline"): {
        "bytes": 733440, "files": ("solve_spec.cu", "atoms.cuh", "step.cuh", "cpasync.cuh", "common.cuh",
                                   "cert_records.cuh", "batched.h", "internal.h"),
        "digest": "955cbcb7a06fa863"},
    ("feature8192_d128", "roofline"): {
        "bytes": 269742336 + 3024384, "files": ("solve_spec.cu", "atoms.cuh", "step.cuh", "cpasync.cuh", "common.cuh",
                                                "cert_records.cuh", "batched.h", "internal.h"),
        "digest": "955cbcb7a06fa863"},
    ("feature8192_d128", "roofline_cost"): {
        "bytes": 4309248 + 206549504, "files": ("cost_bf16.cu", "common.cuh"), "digest": "a6c016e0c5144edc"},
    ("colour_batch64_2048", "roofline_adjoint"): {
        "bytes": 1077042000 + 37607936, "files": ("adjoint.cu", "common.cuh"), "digest": "0e70d4c9330dbe0e"},
}


def kernel_digest(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(ROOT, "paper_2103_05857_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(workload, key):
    """Bytes per launch from the ncu capture, or None if the kernel changed since."""
    e = CAPTURED_TRAFFIC.get((workload, key))
    if e is None or e["digest"] != kernel_digest(e["files"]):
        return None
    return e["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="colour4096_fp32")
    ap.add_argument("--variant", default="BCPFW", choices=list(VARIANTS))
    ap.add_argument("--step-rule", default="ELS", choices=["DEC", "ELS"])
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--max-epochs", type=int, default=None)
    ap.add_argument("--cpu-epochs", type=int, default=None, help="oracle sample size (epochs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--instances", type=int, default=None,
                    help="batched workloads: use only the first K instances (small profiling cases)")
    ap.add_argument("--no-variants", action="store_true",
                    help="colour4096_fp32: skip the variant x rho grid; feature8192_d128: skip the plain-form runs")
    ap.add_argument("--no-protocol", action="store_true",
                    help="colour_batch64_2048: skip the 100-step gradient descent on X")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def sm_count():
    """Streaming multiprocessors of the current device, as the device reports them."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_peak_tflops(peaks):
    """CUDA-core FP32 peak from unit counts and the maximum SM clock
    (SMs x 128 lanes x 2 flops per FMA x clock)."""
    return sm_count() * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# Workload settings
# ---------------------------------------------------------------------------
def settings(args):
    w = args.workload
    s = {"variant": args.variant, "step": args.step_rule, "tol": 1e-6, "max_epochs": 6000,
         "precision": "FP32", "cpu_epochs": 48, "cpu_rows": None}
    if w == "colour256_fp64":
        s.update(variant="BCFW", step="DEC", tol=0.0, max_epochs=200, precision="FP64", cpu_epochs=200)
    elif w == "colour_batch512":
        s.update(max_epochs=20000, cpu_epochs=20)
    elif w == "feature8192_d128":
        s.update(max_epochs=20000, precision="FP32_BF16COST", cpu_epochs=10, cpu_rows=512)
    elif w == "colour_batch64_2048":
        s.update(tol=1e-7, max_epochs=20000, cpu_epochs=10)
    if args.tol is not None:
        s["tol"] = args.tol
    if args.max_epochs is not None:
        s["max_epochs"] = args.max_epochs
    if args.cpu_epochs is not None:
        s["cpu_epochs"] = args.cpu_epochs
    return s


def epoch_kernel_name(s, n):
    """The epoch kernel the library runs for these settings (its own dispatch:
    speculative for pairwise steps on d = 3 points with n <= 4096 and on a
    given cost with n <= 8192, pipelined up to n = 8192, else two-phase; FP64 BCFW up to n = 512 runs on one warp;
    other FP64 and BCFW settings keep the dense-row kernel)."""
    if s["precision"] == "FP64" and s["variant"] == "BCFW" and n <= 512 and not s.get("ga"):
        return ("k_epoch_f64w (one warp, m block updates; dense rows, FP32 argmin screen with exact "
                "FP64 decisions, cost in shared memory)")
    if s["precision"] == "FP64" or s["variant"] == "BCFW":
        return "k_epoch (one CTA, m block updates; dense rows)"
    if s["variant"] == "BCAFW":
        return "k_epoch_sparse (one CTA, m block updates; active-set, away steps)"
    if s["precision"] == "FP32_BF16COST" and n <= 8192 and n % 4 == 0:
        return ("k_epoch_spec (one CTA, m block updates; pairwise; given cost: producers stream each row "
                "through a shared-memory ring, the chain keeps the cost at the likely changed columns; "
                "three chain warps in rotation)")
    if s["precision"] != "FP32_BF16COST" and n <= 4096:
        return ("k_epoch_spec (one CTA, m block updates; pairwise; segment minima and away statistics taken "
                "ahead by producer warps, three chain warps in rotation)")
    if n <= 8192:
        return "k_epoch_pipe (one CTA, m block updates; active-set, pairwise, two control warps)"
    return "k_epoch_sparse (one CTA, m block updates; active-set, pairwise)"


def load(name):
    from paper_2103_05857_gb300 import workloads as W
    x = W.workload(name)
    if isinstance(x, list):
        return [i.rounded() for i in x]
    return x if name == "colour256_fp64" else x.rounded()


def oracle_sample(insts, s):
    """The FP64 oracle as written (single thread) on a bounded sample of the
    workload: `cpu_epochs` epochs of the first instance (for the feature
    workload, of its first `cpu_rows` rows against all n columns: a block
    update's cost depends on n only). Returns (updates, seconds, text)."""
    from oracle import oracle as O
    O.build()
    inst = insts[0] if isinstance(insts, list) else insts
    X, a = inst.X, inst.a
    if s["cpu_rows"]:
        X, a = X[: s["cpu_rows"]], a[: s["cpu_rows"]]
    t0 = time.perf_counter()
    C = O.cost(X, inst.Y)
    _, res, *_ = O.solve(C, a, inst.b, rho=inst.rho, variant=VARIANTS[s["variant"]],
                         step=1 if s["step"] == "ELS" else 0, max_epochs=s["cpu_epochs"], gap_every=1)
    dt = time.perf_counter() - t0
    text = (f"{s['cpu_epochs']} epochs ({res['updates']} block updates) of {s['variant']}-{s['step']} "
            f"on a {len(a)} x {inst.n} instance of the workload, FP64 oracle incl. cost and "
            f"certificates, {dt:.1f} s on 1 of {cpu_cores()} host cores")
    return res["updates"], dt, text


def metric_for(s):
    if s["tol"] > 0:
        return f"block-updates/s to rel. duality gap {s['tol']:g}"
    return f"block-updates/s over {s['max_epochs']} epochs"


def config_for(args, s, insts, ws):
    """The `config` object of both arms' JSON lines."""
    cfg = {"workload": args.workload, "variant": f"{s['variant']}-{s['step']}", "order": "cyclic",
           "precision": s["precision"], "tol_rel_gap": s["tol"], "max_epochs": s["max_epochs"],
           "certificate": ("exact (Thm 2); the library takes it when the gap's geometric decay predicts the "
                           "tolerance (1 to 8 epochs apart), the oracle every epoch"),
           "l2": "flushed (256 MB write) between steps"}
    if isinstance(insts, list):
        cfg.update(instances=len(insts), m_range=[min(i.m for i in insts), max(i.m for i in insts)],
                   n_range=[min(i.n for i in insts), max(i.n for i in insts)], d=3, rho=insts[0].rho,
                   backward=args.workload == "colour_batch64_2048", parallelism=f"lpt{ws}")
    else:
        cfg.update(m=insts.m, n=insts.n, d=int(insts.X.shape[1]), rho=insts.rho, parallelism=f"replicas{ws}")
    return cfg


# ---------------------------------------------------------------------------
# CPU-baseline leg, second part: the FP64 oracle certifies plans the GPU
# returned (outside every timed region; rank 0 only; skipped with
# --no-cpu-baseline). The oracle's certificate (Thm 2) of a plan bounds its
# distance to the optimum, and the stored optimal values (written by
# tests/golden/make_optima.py from the oracle alone) give f* itself.
# ---------------------------------------------------------------------------
def golden_optima(workload):
    p = os.path.join(ROOT, "tests", "golden", f"{workload}_optima.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        return json.load(fh)["optima"]


class OracleCheck:
    def __init__(self, inst, workload):
        from oracle import oracle as O
        O.build()
        self.O = O
        self.inst = inst
        self.C = O.cost(inst.X, inst.Y)
        self.optima = golden_optima(workload)

    def __call__(self, T_dev, rho, reported):
        Th = T_dev.detach().to("cpu").double().numpy()
        c = self.O.certificate(self.C, self.inst.a, self.inst.b, rho, Th)
        out = {"rel_gap": c["g"] / c["f"], "objective": c["f"],
               "library_objective_rel_err": abs(reported["objective"] - c["f"]) / abs(c["f"])}
        opt = self.optima.get(f"{rho:g}")
        if opt:
            out["f_star"] = opt["f"]
            out["objective_vs_f_star"] = (c["f"] - opt["f"]) / opt["f"]
        return out


def colour256_checks(h, S, inst, s, T, X, Y, reported):
    """colour256_fp64: the oracle's own run of the same solve (BCFW with the
    decay rule, cyclic, FP64) must give the GPU's plan bit for bit; and the
    paper's metrics (v) and (vi) of that plan against the exact LP plan T*_LP
    (the oracle's LP solve), computed on the GPU by sr_ot_lp_metrics and
    checked against the oracle's own evaluation."""
    import torch
    from oracle import oracle as O
    O.build()
    C = O.cost(inst.X, inst.Y)
    To, ro, *_ = O.solve(C, inst.a, inst.b, rho=inst.rho, variant=VARIANTS[s["variant"]],
                         step=1 if s["step"] == "ELS" else 0, max_epochs=s["max_epochs"])
    Tg = T.detach().cpu().numpy()
    out = {"plan_bit_identical": bool(np.array_equal(Tg, To)), "max_abs_plan_diff": float(np.abs(Tg - To).max()),
           "objective_rel_err": abs(reported["objective"] - ro["f"]) / abs(ro["f"])}
    L = O.transport_lp(C, inst.a, inst.b)
    g = h.lp_metrics(T, torch.as_tensor(L, dtype=torch.float64, device=T.device), X=X, Y=Y, precision=S.FP64)
    o = O.lp_metrics(C, Tg, L)
    out["lp_metrics"] = {"e_m": g["e_m"], "e_v": g["e_v"], "lp_value": g["lp_value"],
                         "e_m_rel_err_vs_oracle": abs(g["e_m"] - o["e_m"]) / o["e_m"],
                         "e_v_abs_err_vs_oracle": abs(g["e_v"] - o["e_v"]),
                         "reference": "T*_LP of the unrelaxed problem, oracle LP solve (Sec. 5, metrics v, vi)"}
    return out


def feature_checks(inst, T, reported):
    """feature8192_d128: the oracle's certificate (Thm 2, FP64) of the GPU's
    plan under the cost the library approximates -- the squared distances of
    the BF16-rounded points -- and under the exact inputs' cost (the error of
    the mixed-precision form against the FP64 problem)."""
    from oracle import oracle as O
    from paper_2103_05857_gb300 import workloads as W
    O.build()
    Tg = T.detach().to("cpu").double().numpy()
    exact = W.workload("feature8192_d128")
    out = {}
    for key, X, Y in (("bf16_rounded_inputs", W.bf16_round(inst.X), W.bf16_round(inst.Y)),
                      ("exact_inputs", exact.X, exact.Y)):
        C = O.cost(X, Y)
        c = O.certificate(C, inst.a, inst.b, inst.rho, Tg)
        out[key] = {"rel_gap": c["g"] / c["f"], "objective": c["f"],
                    "library_objective_rel_err": abs(reported["objective"] - c["f"]) / abs(c["f"])}
        del C
    return out


# The variant grid on colour4096_fp32: plain BCFW and the paper's three fast
# variants (Sec. 4: away steps, pairwise steps, gap-adaptive sampling), each
# with the exact line search, plus pairwise steps in the paper's default
# uniform order, for rho in {1, 10, 100}; each run to rel. gap 1e-6 or its
# epoch cap (then the gap reached is reported).
VARIANT_GRID = [  # label, variant, order, extra options, epoch cap
    ("BCFW-ELS", "BCFW", "CYCLIC", {}, 600),
    ("BCAFW-ELS", "BCAFW", "CYCLIC", {}, 3000),
    ("BCPFW-ELS", "BCPFW", "CYCLIC", {}, 6000),
    ("BCFW-GAS-ELS", "BCFW", "GAP_ADAPTIVE", {"ga_global_only": 1}, 600),
    ("BCPFW-U-ELS", "BCPFW", "UNIFORM", {}, 6000),
]
GRID_RHOS = (1.0, 10.0, 100.0)


def plain_forms(h, S, inst, X, Y, a, b, stream, flush, mixed_s):
    """feature8192_d128: the plain GPU form beside the mixed-precision one --
    the FP32 cost built on the CUDA cores (no tensor cores, no BF16 rounding)
    with plain BCFW (exact line search), to rel. gap 1e-6 or its epoch cap;
    and, to separate the two effects, the same FP32 cost with pairwise steps.
    Time to the tolerance (or to the cap) with CUDA events, outside the timed
    region of the line."""
    import torch
    out = {"mixed_form_s": mixed_s}
    for label, var, cap in (("plain_bcfw_fp32_cost", "BCFW", 300), ("bcpfw_fp32_cost", "BCPFW", 2000)):
        T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device=X.device)
        opts = S.options(variant=VARIANTS[var], step=S.ELS, order=S.CYCLIC, precision=S.FP32, rho=inst.rho,
                         tol_rel_gap=1e-6, max_epochs=cap, gap_every=1, refresh_every=1)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = h.solve(a, b, T, X=X, Y=Y, opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        out[label] = {"converged": r["status"] == S.OK, "seconds": sec, "epochs": r["epochs"],
                      "rel_gap": r["rel_gap"], "epoch_cap": cap,
                      "mixed_form_speedup": sec / mixed_s if mixed_s > 0 else None}
        del T
    out["note"] = ("seconds = time to rel. gap 1e-6 when converged, else to the epoch cap; the mixed form: BF16 "
                   "tensor-core cost (FP32 accumulation, exact norms) + BCPFW-ELS, the timed step of this line")
    return out


def variant_grid(h, S, inst, X, Y, a, b, T, stream, flush, check):
    import torch
    cells = []
    for label, var, order, extra, cap in VARIANT_GRID:
        for rho in GRID_RHOS:
            opts = S.options(variant=VARIANTS[var], step=S.ELS, order=getattr(S, order), precision=S.FP32,
                             rho=rho, tol_rel_gap=1e-6, max_epochs=cap, gap_every=1, refresh_every=1,
                             seed=7, **extra)
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = h.solve(a, b, T, X=X, Y=Y, opts=opts)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            cell = {"variant": label, "rho": rho, "converged": r["status"] == S.OK, "seconds": sec,
                    "epochs": r["epochs"], "rel_gap": r["rel_gap"],
                    "block_updates_per_s": r["block_updates"] / sec}
            if check is not None:
                cell["oracle_check"] = check(T, rho, r)
            cells.append(cell)
    return {"workload": "colour4096_fp32", "tol_rel_gap": 1e-6, "step": "ELS", "seed": 7,
            "note": "seconds = time to the tolerance when converged, else to the epoch cap (rel_gap then "
                    "is the gap reached)", "cells": cells}


# ---------------------------------------------------------------------------
def bench_reference(args, ws, rank):
    """The oracle timed on the host cores: K steps, each a bounded sample."""
    if rank != 0:
        return
    s = settings(args)
    insts = load(args.workload)
    small = dict(s)
    small["cpu_epochs"] = 1
    oracle_sample(insts, small)
    tot_u, tot_s, text = 0, 0.0, ""
    for _ in range(args.steps):
        u, dt, text = oracle_sample(insts, s)
        tot_u += u
        tot_s += dt
    v = tot_u / tot_s
    line = {
        "impl": "reference", "metric": metric_for(s), "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_for(args, s, insts, ws),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": text},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class Harness:
    """Warm-up, timed steps (CUDA events on the handle's stream, L2 flushed
    before each step, barrier + synchronize on both sides), clocks, launches."""

    def __init__(self, h, dev, stream, ws):
        import torch
        self.torch = torch
        self.h, self.dev, self.stream, self.ws = h, dev, stream, ws
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def run(self, step, steps, warmup, profile_kinds=()):
        torch = self.torch
        for _ in range(warmup):
            step()
        torch.cuda.synchronize(self.dev)
        clocks = ClockSampler(self.dev.index)
        clocks.start()
        self.h.profile(True)
        l0 = self.h.launch_count()
        out, ms = [], []
        for _ in range(steps):
            self.flush.zero_()
            barrier(self.ws)
            torch.cuda.synchronize(self.dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            out.append(step())
            e1.record(self.stream)
            torch.cuda.synchronize(self.dev)
            ms.append(e0.elapsed_time(e1))
        barrier(self.ws)
        launches = self.h.launch_count() - l0
        prof = {k: self.h.profile_read(k) for k in profile_kinds}
        self.h.profile(False)
        return out, ms, launches, prof, clocks.stop()

    def e2e(self, step_with_copies, steps):
        torch = self.torch
        ms = []
        for _ in range(steps):
            self.flush.zero_()
            barrier(self.ws)
            torch.cuda.synchronize(self.dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            step_with_copies()
            e1.record(self.stream)
            torch.cuda.synchronize(self.dev)
            ms.append(e0.elapsed_time(e1))
        return ms


def alu_roofline(flops, avg_ms, peaks, peak_src, kernel, extra=None):
    peak = fp32_peak_tflops(peaks)
    achieved = flops / (avg_ms / 1e3) / 1e12
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
         "traffic": None, "peak_source": f"derived: {sm_count()} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                        f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_src} clock)",
         "kernel": kernel, "avg_launch_ms": avg_ms}
    if extra:
        r.update(extra)
    return r


def hbm_roofline(nbytes, avg_ms, peaks, peak_src, kernel, extra=None):
    achieved = nbytes / (avg_ms / 1e3) / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
         "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_src,
         "kernel": kernel, "avg_launch_ms": avg_ms}
    if extra:
        r.update(extra)
    return r


def bench_single(args, s, ws, rank, local, cpu_leg):
    """One instance per rank (replicas): colour4096_fp32, colour256_fp64,
    feature8192_d128."""
    import torch
    from paper_2103_05857_gb300 import sr_ot as S

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    inst = load(args.workload)
    m, n, d = inst.m, inst.n, inst.X.shape[1]
    fp64 = s["precision"] == "FP64"
    dt = torch.float64 if fp64 else torch.float32
    npdt = np.float64 if fp64 else np.float32
    stream = torch.cuda.current_stream(dev)
    h = S.Handle(local, stream)
    H = Harness(h, dev, stream, ws)

    hX, hY, ha, hb = (torch.from_numpy(np.ascontiguousarray(v, dtype=npdt)).pin_memory()
                      for v in (inst.X, inst.Y, inst.a, inst.b))
    hT = torch.empty((m, n), dtype=dt).pin_memory()
    X, Y, a, b = (t.to(dev) for t in (hX, hY, ha, hb))
    T = torch.zeros((m, n), dtype=dt, device=dev)
    opts = S.options(variant=VARIANTS[s["variant"]], step=1 if s["step"] == "ELS" else 0, order=S.CYCLIC,
                     precision=getattr(S, s["precision"]), rho=inst.rho, tol_rel_gap=s["tol"],
                     max_epochs=s["max_epochs"], gap_every=1, refresh_every=1,
                     cert_schedule=1 if s["tol"] > 0 else 0)

    def step():
        return h.solve(a, b, T, X=X, Y=Y, opts=opts)

    out, ms, launches, prof, clk = H.run(step, args.steps, args.warmup,
                                         (S.PROF_EPOCH, S.PROF_CERT, S.PROF_COST))
    updates = sum(r["block_updates"] for r in out)
    from paper_2103_05857_gb300.shard import gather_max
    tot_max = gather_max(sum(ms), ws)
    value = updates * ws / (tot_max / 1e3)

    def step_e2e():
        X.copy_(hX, non_blocking=True)
        Y.copy_(hY, non_blocking=True)
        a.copy_(ha, non_blocking=True)
        b.copy_(hb, non_blocking=True)
        h.solve(a, b, T, X=X, Y=Y, opts=opts)
        hT.copy_(T, non_blocking=True)

    e2e_ms = H.e2e(step_e2e, args.steps)
    e2e_value = updates * ws / (gather_max(sum(e2e_ms), ws) / 1e3)
    h2d = sum(t.numel() * t.element_size() for t in (hX, hY, ha, hb))
    d2h = hT.numel() * hT.element_size()

    peaks, peak_src = measured_peaks()
    ep_ms, ep_n = prof[S.PROF_EPOCH]
    ce_ms, ce_n = prof[S.PROF_CERT]
    co_ms, co_n = prof[S.PROF_COST]
    avg = ep_ms / max(ep_n, 1)
    supp = float((T > 0).sum().item()) / m
    extra = {"launches": ep_n, "chain_ns_per_update": 1e6 * avg / m, "cert_avg_ms": ce_ms / max(ce_n, 1),
             "hbm_bytes_per_update": 8 * supp, "mean_support": supp}
    kname = epoch_kernel_name(s, n)
    if kname.startswith("k_epoch_spec"):
        # the chain alone, with the same hand-over (and with one warp, none)
        floor3 = h.chain_floor(3)
        extra.update(chain_floor_ns=floor3, chain_floor_ns_one_warp=h.chain_floor(1),
                     chain_frac=floor3 / extra["chain_ns_per_update"])
    if s["precision"] == "FP32_BF16COST":
        # the epoch reads the materialised cost: one row of C (4 n bytes) per
        # block update, and the changed plan entries (8 bytes per support entry)
        roof = hbm_roofline(float(m) * (4.0 * n + 8.0 * supp), avg, peaks, peak_src, kname, extra)
    else:
        roof = alu_roofline(FLOPS_PER_GRAD * n * m, avg, peaks, peak_src, kname, extra)
    cfg = config_for(args, s, inst, ws)
    line = {"metric": metric_for(s),
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic", "config": cfg,
            "time_to_gap_s": tot_max / args.steps / 1e3,
            "epochs_per_solve": [r["epochs"] for r in out],
            "final_rel_gap": [r["rel_gap"] for r in out],
            "converged": all(r["status"] == 0 for r in out),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "clocks": clk}
    check = None
    if cpu_leg and args.workload == "colour4096_fp32":
        check = OracleCheck(inst, args.workload)
        line["oracle_check"] = check(T, inst.rho, out[-1])
    elif cpu_leg and args.workload == "colour256_fp64":
        line["oracle_check"] = colour256_checks(h, S, inst, s, T, X, Y, out[-1])
    elif cpu_leg and args.workload == "feature8192_d128":
        line["oracle_check"] = feature_checks(inst, T, out[-1])
    if args.workload == "colour4096_fp32" and ws == 1 and not args.no_variants:
        line["variants"] = variant_grid(h, S, inst, X, Y, a, b, T, stream, H.flush, check)
    if args.workload == "feature8192_d128" and ws == 1 and not args.no_variants:
        line["vs_plain_gpu"] = plain_forms(h, S, inst, X, Y, a, b, stream, H.flush, line["time_to_gap_s"])
    if co_n:
        co_avg = co_ms / co_n
        line["roofline_cost"] = hbm_roofline(4.0 * m * n + 4.0 * (m + n) * d + 2.0 * (m + n) * d, co_avg,
                                             peaks, peak_src, "k_round_bf16 + k_cost_umma (tcgen05)",
                                             {"tflops_bf16": 2.0 * m * n * d / (co_avg / 1e3) / 1e12})
    h.close()
    return line, inst


def gd_protocol(h, S, pb, insts, kw, stream, steps=100):
    """The differentiable form in use: 100 steps of gradient descent on the
    source points X of the whole batch, X <- X - lr dX with dX the envelope
    gradient (sr_ot_grad_batched) at the current plans, each step followed by
    a batched solve warm-started from the previous plans (batch_warm_start).
    lr = 0.005 m moves every x_i 1 % of the way to its barycentric projection
    (dX_i = 2 a_i (x_i - x^_i), a_i = 1/m), i.e. gradient descent on the sum
    of the instances' optimal values, which must not increase."""
    import torch
    m = insts[0].m
    lr = 0.005 * m
    X = pb.X.clone()
    T = pb.T  # converged plans of the timed solves
    _, res0 = h.solve_batched(X, pb.Y, pb.a, pb.b, T, pb.sizes, pb.offsets, batch_warm_start=1, **kw)
    vals = [sum(r["objective"] for r in res0)]
    epochs, conv = [], True
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g = h.grad_batched(X, pb.Y, pb.b, T, pb.sizes, pb.offsets, want=("dX",), rho=insts[0].rho,
                           precision=S.FP32)
        X.sub_(lr * g["dX"])
        _, res = h.solve_batched(X, pb.Y, pb.a, pb.b, T, pb.sizes, pb.offsets, batch_warm_start=1, **kw)
        vals.append(sum(r["objective"] for r in res))
        epochs.append(float(np.median([r["epochs"] for r in res])))
        conv = conv and all(r["status"] == 0 for r in res)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    incr = [b - a for a, b in zip(vals, vals[1:])]
    return {"steps": steps, "lr": lr, "objective_sum_start": vals[0], "objective_sum_end": vals[-1],
            "non_increasing_steps": sum(d <= 1e-6 * abs(vals[0]) for d in incr), "seconds": sec,
            "ms_per_step": 1e3 * sec / steps, "warm_solve_epochs_median": float(np.median(epochs)),
            "all_converged": conv,
            "note": "each step: adjoint at the current plans, X update, batched solve warm-started from them"}


def bench_batch(args, s, ws, rank, local):
    """colour_batch512 and colour_batch64_2048: this rank's share of the
    instances in one persistent launch (plus the adjoint for the latter)."""
    import torch
    from paper_2103_05857_gb300 import sr_ot as S
    from paper_2103_05857_gb300.batch import PackedBatch
    from paper_2103_05857_gb300.shard import gather_max, gather_sum, lpt_partition

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    allinst = load(args.workload)
    if args.instances:
        allinst = allinst[: args.instances]
    share = lpt_partition([i.m * i.n for i in allinst], ws)[rank]
    insts = [allinst[k] for k in share]
    stream = torch.cuda.current_stream(dev)
    h = S.Handle(local, stream)
    H = Harness(h, dev, stream, ws)
    pb = PackedBatch(insts, device=dev, pin=True)
    hT = torch.empty(pb.total_T, dtype=torch.float32).pin_memory()
    kw = dict(variant=VARIANTS[s["variant"]], step=1 if s["step"] == "ELS" else 0, rho=insts[0].rho,
              tol_rel_gap=s["tol"], max_epochs=s["max_epochs"], gap_every=1)
    backward = args.workload == "colour_batch64_2048"

    def step():
        st, res = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, **kw)
        if backward:
            h.grad_batched(pb.X, pb.Y, pb.b, pb.T, pb.sizes, pb.offsets, rho=insts[0].rho, precision=S.FP32)
        return res

    out, ms, launches, prof, clk = H.run(step, args.steps, args.warmup, (S.PROF_BATCH, S.PROF_GRAD))
    updates = sum(r["block_updates"] for res in out for r in res)
    tot_max = gather_max(sum(ms), ws)
    updates_all = gather_sum(updates, ws)
    value = updates_all / (tot_max / 1e3)

    def step_e2e():
        pb.X.copy_(pb.hX, non_blocking=True)
        pb.Y.copy_(pb.hY, non_blocking=True)
        pb.a.copy_(pb.ha, non_blocking=True)
        pb.b.copy_(pb.hb, non_blocking=True)
        step()
        hT.copy_(pb.T, non_blocking=True)

    e2e_ms = H.e2e(step_e2e, args.steps)
    e2e_value = updates_all / (gather_max(sum(e2e_ms), ws) / 1e3)
    h2d = sum(t.numel() * 4 for t in (pb.hX, pb.hY, pb.ha, pb.hb))
    d2h = hT.numel() * 4

    peaks, peak_src = measured_peaks()
    b_ms, b_n = prof[S.PROF_BATCH]
    flops = FLOPS_PER_GRAD * sum(r["block_updates"] * insts[k].n for res in out for k, r in enumerate(res))
    # the makespan is set by the instance with the most block updates: its
    # mean time per update if it ran from the first to the last moment
    longest = max(r["block_updates"] for r in out[-1])
    batch_ms = b_ms / max(b_n, 1)
    floor3 = h.chain_floor(3)
    kname = ("k_spec_batch_init + k_epoch_spec in batch mode (one CTA per instance for the whole solve: "
             "speculative epochs, certificate inside the CTA)" if s["variant"] == "BCPFW"
             else "k_batched (persistent, one CTA per instance at a time)")
    roof = alu_roofline(flops / max(len(out), 1), batch_ms, peaks, peak_src, kname,
                        {"launches": b_n, "instances": len(insts), "longest_chain_updates": longest,
                         "longest_chain_ns_per_update": 1e6 * batch_ms / longest,
                         "chain_floor_ns": floor3, "chain_frac": floor3 / (1e6 * batch_ms / longest)})
    res0 = out[-1]
    line = {"metric": metric_for(s),
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": config_for(args, s, allinst, ws),
            "converged": sum(r["status"] == 0 for r in res0), "instances_on_rank0": len(insts),
            "epochs_max": max(r["epochs"] for r in res0), "epochs_median": float(np.median([r["epochs"] for r in res0])),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "clocks": clk}
    # the plain GPU form: the same instances solved one after another on the
    # single-instance path (sr_ot_solve, same rule and tolerance; with the
    # backward pass, sr_ot_grad after each): evenly spaced instances,
    # extrapolated to the whole share by their block updates
    if True:
        nsamp = 8 if backward else 32
        sample = list(range(0, len(insts), max(1, len(insts) // nsamp)))[:nsamp]
        seq_upd, seq_ms = 0, 0.0
        for k in sample:
            inst = insts[k]
            Xs, Ys = (torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32, device=dev) for v in (inst.X, inst.Y))
            as_, bs = (torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32, device=dev) for v in (inst.a, inst.b))
            Ts = torch.zeros((inst.m, inst.n), dtype=torch.float32, device=dev)
            h.solve(as_, bs, Ts, X=Xs, Y=Ys, precision=S.FP32, max_epochs=1, **{kk: vv for kk, vv in kw.items() if kk != "max_epochs"})
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = h.solve(as_, bs, Ts, X=Xs, Y=Ys, precision=S.FP32, **kw)
            if backward:
                h.grad(Ts, X=Xs, Y=Ys, b=bs, precision=S.FP32, rho=insts[0].rho)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            seq_ms += e0.elapsed_time(e1)
            seq_upd += r["block_updates"]
        seq_rate = seq_upd / (seq_ms / 1e3)
        line["sequential_baseline"] = {
            "value": seq_rate, "unit": UNIT,
            "sample": f"{len(sample)} of {len(insts)} instances solved one after another with sr_ot_solve"
                      f"{' and sr_ot_grad' if backward else ''} ({s['variant']}-{s['step']}, same tolerance), "
                      f"{seq_ms / 1e3:.2f} s for {seq_upd} block updates",
            "extrapolated_s": (updates / len(out)) / seq_rate,
            "batched_speedup": value / seq_rate}
    if backward and ws == 1 and not args.no_protocol:
        line["gd_100"] = gd_protocol(h, S, pb, insts, kw, stream)
    g_ms, g_n = prof[S.PROF_GRAD]
    if g_n:
        tbytes = 4.0 * pb.total_T + 4.0 * sum(3 * (i.m + i.n) * 2 + i.n * 2 for i in insts)
        line["roofline_adjoint"] = hbm_roofline(tbytes, g_ms / g_n, peaks, peak_src,
                                                "k_adj_tiles + k_adj_finish", {"launches": g_n})
    if backward:
        # colour-transfer tail over the same plans (barycentric projection,
        # e_c, sparsity; Sec. 5.1 and 5): device time of the library's own
        # launches, outside the timed solve
        h.profile(True)
        for _ in range(4):
            _, tstats = h.transfer_batched(pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, precision=S.FP32,
                                           xhat_numel=pb.X.numel())
        t_ms, t_n = h.profile_read(S.PROF_GRAD)
        h.profile(False)
        tb = 4.0 * pb.total_T + 4.0 * sum(3 * i.n + i.n + i.m + 3 * i.m for i in insts)
        line["roofline_transfer"] = hbm_roofline(
            tb, t_ms / max(t_n, 1), peaks, peak_src, "k_adj_tiles + k_adj_finish + k_transfer_stats",
            {"launches": t_n, "e_c_max": max(t["e_c"] for t in tstats),
             "sparsity_mean": float(np.mean([t["sparsity"] for t in tstats]))})
    h.close()
    return line, allinst


def bench_ours(args, ws, rank, local):
    s = settings(args)
    cpu_leg = rank == 0 and not args.no_cpu_baseline
    if args.workload in BATCH_WORKLOADS:
        line, insts = bench_batch(args, s, ws, rank, local)
    else:
        line, insts = bench_single(args, s, ws, rank, local, cpu_leg)
    for key in ("roofline", "roofline_cost", "roofline_adjoint", "roofline_transfer"):
        if key in line:
            line[key]["traffic"] = captured_traffic(args.workload, key)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            u, dt, text = oracle_sample(insts, s)
            cpu = {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": text}
        line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    return line


def main():
    args = parse()
    ws, rank, local = dist_setup()
    args.gpus = ws
    try:
        if args.impl == "reference":
            bench_reference(args, ws, rank)
        else:
            bench_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
