"""Write the stored expected values under tests/golden/ from the FP64 oracle only.

qn2d_n63_seed0.json: the 2-D 63x63 manufactured problem (-Lap u + u^3 = f,
Dirichlet 0, second-order differences, Sec. 3.2; quasi-Newton of Sec. 4
eq. identity-method with the paper's beta rule), seed 0, zero start, tolerance
1e-10 on ||F||/||f||: iteration count, relative-residual history and the
converged solution at a fixed set of nodes.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2502_03611_gb300.inputs import manufactured_problem  # noqa: E402


def main():
    n, seed = 63, 0
    _, f = manufactured_problem(n, 2, seed=seed)
    U, hist, ok = O.qn_solve(f, tol=1e-10)
    assert ok
    idx = [(0, 0), (5, 17), (31, 31), (40, 2), (62, 62), (10, 50)]
    out = {
        "source": "oracle.qn_solve (FP64 numpy), written by tests/golden/make_golden.py",
        "problem": "2-D -Lap u + u^3 = f, manufactured u* (4x4 sine modes, amp 0.1), Sec. 3.2 / Sec. 4",
        "n": n, "seed": seed, "tol": 1e-10,
        "iterations": len(hist) - 1,
        "rel_history": [h["rel"] for h in hist],
        "beta_history": [h["beta"] for h in hist],
        "sample_index": idx,
        "sample_value": [float(U[y, x]) for (y, x) in idx],
    }
    with open(os.path.join(HERE, "qn2d_n63_seed0.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
