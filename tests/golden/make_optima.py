"""Write the FP64 oracle's optimal values of the colour4096_fp32 workload.

The semi-relaxed problem has a unique optimal value f* (f is strictly convex
in the column sums and linear in T, Sec. 3), so a converged solve of any
variant must reach it. This script runs only the oracle (BCPFW with the
exact line search, Alg. A.3 and eq. 10, FP64, cyclic order) on the float32
rounding of the workload's inputs -- the exact values the FP32 library sees
-- until the duality gap (Thm 2) is below a tolerance times the objective,
for each penalty weight rho in {1, 10, 100} (one process each), and stores f
and g of the final plan: f* lies in [f - g, f]. The tolerance is 1e-9 for
rho = 1 and 10 and 1e-7 for rho = 100, where the oracle's pairwise steps
need tens of thousands of epochs below that; a 1e-7 interval is still far
inside the 1.2e-6 the tests check against.

    python tests/golden/make_optima.py     (about 20 minutes on three cores)
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "colour4096_fp32_optima.json")
TOLS = {1.0: 1e-9, 10.0: 1e-9, 100.0: 1e-7}
RHOS = tuple(TOLS)


def optimum(rho):
    from oracle import oracle as O
    from paper_2103_05857_gb300 import workloads as W
    inst = W.workload("colour4096_fp32").rounded()
    C = O.cost(inst.X, inst.Y)
    t0 = time.time()
    _, r, *_ = O.solve(C, inst.a, inst.b, rho=rho, variant=O.BCPFW, step=O.ELS, order=O.CYCLIC,
                       tol_rel_gap=TOLS[rho], max_epochs=200000, gap_every=10)
    assert r["converged"], r
    print(f"rho={rho:g}: f={r['f']!r} g={r['g']:.3e} epochs={r['epochs']} ({time.time() - t0:.0f} s)", flush=True)
    return rho, {"f": r["f"], "g": r["g"], "f_lower": r["f"] - r["g"], "epochs": int(r["epochs"]),
                 "tol_rel_gap": TOLS[rho]}


def main():
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    O.build()
    with mp.get_context("spawn").Pool(len(RHOS)) as pool:
        res = dict(pool.map(optimum, RHOS))
    out = {"workload": "colour4096_fp32 (float32-rounded inputs), squared-Euclidean cost",
           "solver": "oracle BCPFW-ELS, cyclic, FP64, stopped at g <= tol_rel_gap f",
           "optima": {f"{rho:g}": res[rho] for rho in RHOS}}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
