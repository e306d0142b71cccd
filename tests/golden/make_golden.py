"""Writes the oracle's reference flows used by the GPU flow-parity tests.

Calls only the oracle.  Run from the repository root:
    python tests/golden/make_golden.py
Output: tests/golden/flow_cfg1.npz (cfg1 workload: t'=-0.25, mu=4t', U=3,
8x8 coarse grid, Nff=5, 96x96 fine grid, Lambda0=10, threshold 50,
DoPri5 rtol=1e-8 atol=1e-10) with Lambda_c, classification and the state at
the checkpoints Lambda = 1, 0.3, 0.1, 0.05.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import flow as fl  # noqa: E402
from oracle.model import Problem  # noqa: E402

CHECKPOINTS = (1.0, 0.3, 0.1, 0.05)


def main():
    c = W.config("cfg1")
    prob = Problem(c["t"], c["tp"], c["mu"], c["U"], W.bonds_for_shells(c["shells"]),
                   c["nc"], c["nc"], c["nf"], c["nf"]).check()
    res = fl.flow(prob, c["lambda0"], c["lambda_min"], c["threshold"], rtol=1e-8,
                  atol=1e-10, h0=-0.05, checkpoints=CHECKPOINTS)
    cls = res.classification
    np.savez_compressed(
        os.path.join(HERE, "flow_cfg1.npz"),
        lambda_c=res.lambda_c, diverged=res.diverged, n_rhs=res.n_rhs,
        n_accepted=res.n_accepted, n_rejected=res.n_rejected,
        channel=cls["channel"], l_index=cls["l_index"], m=cls["m"], n=cls["n"],
        y_c=res.y, checkpoints=np.array(CHECKPOINTS),
        y_checkpoints=np.stack([res.checkpoints[k] for k in CHECKPOINTS]))
    print(res.lambda_c, cls, res.n_rhs, res.n_accepted, res.n_rejected)


if __name__ == "__main__":
    main()
