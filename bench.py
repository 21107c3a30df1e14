"""Benchmark: block-coordinate Frank-Wolfe solves of semi-relaxed OT on GB300.

One step = one complete solve of the colour4096_fp32 workload (m = n = 4096
RGB-like points from seeded 8-component Gaussian mixtures, Dirichlet(1)
target weights, rho = 10, squared-Euclidean cost on the fly) to relative
duality gap 1e-6, with the certificate (Thm 2) taken every epoch. `value` is
block updates per second over the timed solves; `ms_per_step` is the time to
gap. Inputs are resident in HBM when the timed region starts; L2 is flushed
(256 MB write) between timed solves.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun with N > 1, every rank solves its own independent replica
(a single solve does not shard: each block update reads the residual the
previous one wrote); value = all ranks' block updates / max rank time.
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

METRIC = "block-updates/s to rel. duality gap 1e-6"
UNIT = "block-updates/s"
VARIANTS = {"BCFW": 0, "BCAFW": 1, "BCPFW": 2}
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="colour4096_fp32")
    ap.add_argument("--variant", default="BCPFW", choices=list(VARIANTS))
    ap.add_argument("--step-rule", default="ELS", choices=["DEC", "ELS"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-epochs", type=int, default=6000)
    ap.add_argument("--cpu-epochs", type=int, default=48, help="oracle sample size (epochs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


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


def load_instance(name):
    from paper_2103_05857_gb300 import workloads as W
    return W.workload(name).rounded()


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_oracle_sample(inst, variant, step_rule, epochs):
    """The FP64 oracle (single thread, as written) on `epochs` epochs of the
    same workload, certificate every epoch. Returns (updates, seconds)."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    C = O.cost(inst.X, inst.Y)
    _, res, *_ = O.solve(C, inst.a, inst.b, rho=inst.rho, variant=VARIANTS[variant],
                         step=1 if step_rule == "ELS" else 0, max_epochs=epochs, gap_every=1)
    return res["updates"], time.perf_counter() - t0


# ---------------------------------------------------------------------------
def bench_reference(args, ws, rank):
    """The oracle timed on the host cores: K steps, each a bounded sample."""
    if rank != 0:
        return
    inst = load_instance(args.workload)
    ep = max(1, args.cpu_epochs // 4)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        run_oracle_sample(inst, args.variant, args.step_rule, 1)
    tot_u, tot_s = 0, 0.0
    for _ in range(args.steps):
        u, s = run_oracle_sample(inst, args.variant, args.step_rule, ep)
        tot_u += u
        tot_s += s
    v = tot_u / tot_s
    sample = (f"{ep} epochs ({ep * inst.m} block updates) of {args.variant}-{args.step_rule} "
              f"on {args.workload} per step, FP64 oracle, certificate every epoch")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "m": inst.m, "n": inst.n, "rho": inst.rho,
                   "variant": args.variant, "step_rule": args.step_rule},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_ours(args, ws, rank, local):
    import torch
    from paper_2103_05857_gb300 import sr_ot as S

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    inst = load_instance(args.workload)
    m, n = inst.m, inst.n
    stream = torch.cuda.current_stream(dev)
    h = S.Handle(local, stream)

    # pinned host copies (for the end-to-end leg) and resident device copies
    hX = torch.from_numpy(inst.X.astype(np.float32)).pin_memory()
    hY = torch.from_numpy(inst.Y.astype(np.float32)).pin_memory()
    ha = torch.from_numpy(inst.a.astype(np.float32)).pin_memory()
    hb = torch.from_numpy(inst.b.astype(np.float32)).pin_memory()
    hT = torch.empty((m, n), dtype=torch.float32).pin_memory()
    X, Y, a, b = (t.to(dev) for t in (hX, hY, ha, hb))
    T = torch.zeros((m, n), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    opts = S.options(variant=VARIANTS[args.variant], step=1 if args.step_rule == "ELS" else 0,
                     order=S.CYCLIC, precision=S.FP32, rho=inst.rho, tol_rel_gap=args.tol,
                     max_epochs=args.max_epochs, gap_every=1, refresh_every=1)

    def solve_once():
        return h.solve(a, b, T, X=X, Y=Y, opts=opts)

    for _ in range(args.warmup):
        solve_once()
    torch.cuda.synchronize(dev)

    # ---- timed region: inputs resident in HBM --------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    h.profile(True)
    launches0 = h.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    for k in range(args.steps):
        flush.zero_()
        barrier(ws)
        torch.cuda.synchronize(dev)
        ev[k][0].record(stream)
        results.append(solve_once())
        ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    launches = h.launch_count() - launches0
    ep_ms, ep_groups = h.profile_read(S.PROF_EPOCH)
    ce_ms, ce_groups = h.profile_read(S.PROF_CERT)
    h.profile(False)
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    tot_ms = sum(step_ms)
    updates = sum(r["block_updates"] for r in results)
    tot_ms_max = allreduce_max(tot_ms, ws)
    updates_all = updates * ws
    value = updates_all / (tot_ms_max / 1e3)

    # ---- end to end through the public API with host buffers -----------------
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        X.copy_(hX, non_blocking=True)
        Y.copy_(hY, non_blocking=True)
        a.copy_(ha, non_blocking=True)
        b.copy_(hb, non_blocking=True)
        r = h.solve(a, b, T, X=X, Y=Y, opts=opts)
        hT.copy_(T, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append(t0.elapsed_time(t1))
    e2e_updates = updates / args.steps * args.steps
    e2e_value = updates_all / (allreduce_max(sum(e2e_ms), ws) / 1e3)
    h2d = sum(t.numel() * 4 for t in (hX, hY, ha, hb))
    d2h = hT.numel() * 4

    # ---- roofline of the dominant kernel (the epoch kernel) --------------------
    peaks, peak_src = measured_peaks()
    per_update_bytes = 4 * n + 8  # FP32 row of T read once, the two changed entries written
    if args.variant != "BCPFW":
        per_update_bytes = 4 * n + 4 * n  # dense convex combination rewrites the row support
    launch_bytes = per_update_bytes * m
    avg_launch_ms = ep_ms / max(ep_groups, 1)
    achieved = launch_bytes / (avg_launch_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_source": peak_src, "kernel": "k_epoch (one CTA, m block updates)",
                "avg_launch_ms": avg_launch_ms, "launches": ep_groups,
                "cert_avg_ms": ce_ms / max(ce_groups, 1),
                "chain_ns_per_update": 1e6 * avg_launch_ms / m}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            u, s = run_oracle_sample(inst, args.variant, args.step_rule, args.cpu_epochs)
            cpu = {"value": u / s, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_epochs} epochs ({u} block updates) of {args.variant}-"
                             f"{args.step_rule} on {args.workload}, FP64, certificate every epoch, "
                             f"{s:.1f} s on 1 of {cpu_cores()} host cores"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "d": 3, "rho": inst.rho,
                       "variant": f"{args.variant}-{args.step_rule}", "order": "cyclic",
                       "tol_rel_gap": args.tol, "certificate_every_epochs": 1,
                       "parallelism": f"replicas{ws}", "l2": "flushed (256 MB write) between solves"},
            "time_to_gap_s": tot_ms_max / args.steps / 1e3,
            "epochs_per_solve": [r["epochs"] for r in results],
            "final_rel_gap": [r["rel_gap"] for r in results],
            "converged": all(r["status"] == 0 for r in results),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    h.close()
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
