"""Writes tests/golden/p2_oracle.txt: the FP64 oracle's evaluation of the P2 workload (C2's
model and HODLR settings on a 128^2 grid) at two parameter points.

Calls only the oracle (oracle.hodlr.build, oracle.likelihood.evaluate) and the seeded input
generator (synth).  For each theta it records the oracle's per-pair pivot sets (the pivoted
QR of Alg. 1 step 3 with the rank rule max(tol, guard) |R_11|), the NLL, the gradient and the
expected Fisher matrix of the densified K~ (eq. log-like / score / fisher info approximated),
in the layout read by tests/test_gpu_parity_c2.py.  Run from the repository root:
    python tests/golden/make_p2_golden.py
It takes about 15 minutes on 8 cores (two dense 16384 x 16384 evaluations).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import hodlr as oh, likelihood as ol  # noqa: E402
from oracle.physics import Model  # noqa: E402
from oracle.tree import Tree  # noqa: E402

# the configuration's own parameter point (the one y is simulated at, where the score is a
# zero-mean random vector) and a starting point of an optimisation away from it, where every
# score component is large (the two points of the paper's accuracy tables, Sec. 5.2.2)
THETAS = [(1.0, 0.1, 8.0, 1e-4), (1.5, 0.15, 6.0, 2e-4)]


def main(out=os.path.join(os.path.dirname(os.path.abspath(__file__)), "p2_oracle.txt")):
    w = synth.workload("P2")
    m, t = Model(w.dim, w.G, w.nvar, w.nu), Tree(w.dim, w.G, w.nvar, w.leaf)
    y = t.to_tree(synth.simulate_y(w))
    lines = ["# FP64 oracle evaluation of workload P2 (written by tests/golden/make_p2_golden.py)",
             f"# N {t.N} tau {t.tau} leaf {w.leaf} cap {w.cap} c {w.c} tol {w.tol!r} guard {w.guard!r} "
             f"probe seed {w.seed_probe} data seed {w.seed_data}",
             "# per theta: 'theta' 4 values, 'nll', 'grad' 4, 'fisher' 16 (row-major),",
             "# then 'piv <level> <pair> <rank> <J...>' per block pair (pivot sets of the pivoted QR)"]
    for theta in THETAS:
        t0 = time.time()
        H = oh.build(m, t, theta, c=w.c, cap=w.cap, tol=w.tol, guard=w.guard, seed=w.seed_probe)
        f, g, F = ol.evaluate(H, y)
        print(f"theta {theta}: {time.time() - t0:.0f} s, ranks {[max(r) for r in H.ranks()]}", flush=True)
        lines.append("theta " + " ".join(repr(float(v)) for v in theta))
        lines.append(f"nll {f!r}")
        lines.append("grad " + " ".join(repr(float(v)) for v in g))
        lines.append("fisher " + " ".join(repr(float(v)) for v in F.reshape(-1)))
        for l, lvl in enumerate(H.pivots(), start=1):
            for p, J in enumerate(lvl):
                lines.append(f"piv {l} {p} {len(J)} " + " ".join(str(int(j)) for j in J))
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
