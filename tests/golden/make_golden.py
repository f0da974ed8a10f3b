"""Writes tests/golden/tiny_en.json: exact Elastic Net minimisers of small hand-written
problems, computed by exhaustive sign-pattern enumeration (oracle.checkers.brute_force).

The paper prints no worked example, so these fixtures carry the textbook
characterisation of the Elastic Net minimiser (Sec. 1 objective) instead.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import checkers as C  # noqa: E402

CASES = [
    # A is written row by row (m x n); b has length m.
    dict(name="m5n4", A=[[1.0, 0.5, -0.2, 0.0], [0.3, -1.0, 0.8, 0.1], [-0.7, 0.2, 0.4, -1.2],
                         [0.9, 0.9, -0.6, 0.5], [0.0, -0.3, 1.1, 0.7]],
         b=[1.5, -0.8, 0.3, 2.0, -1.1], lam1=0.6, lam2=0.4),
    dict(name="m4n6", A=[[0.2, -1.3, 0.5, 0.9, -0.4, 1.0], [1.1, 0.6, -0.8, 0.3, 0.2, -0.5],
                         [-0.6, 0.4, 1.2, -1.0, 0.8, 0.1], [0.5, -0.2, -0.3, 0.7, 1.4, -0.9]],
         b=[2.0, -1.0, 0.5, 1.2], lam1=0.35, lam2=0.1),
    dict(name="m3n5_ridge_limit", A=[[1.0, 2.0, 0.0, -1.0, 0.5], [0.0, 1.0, 1.0, 2.0, -0.5],
                                     [1.0, -1.0, 2.0, 0.0, 1.0]],
         b=[3.0, -1.0, 2.0], lam1=0.0, lam2=0.5),
    dict(name="m4n3_all_zero", A=[[1.0, 0.0, 0.5], [0.0, 1.0, -0.5], [1.0, 1.0, 0.0], [0.5, -0.5, 1.0]],
         b=[0.2, -0.1, 0.1, 0.3], lam1=5.0, lam2=1.0),
]


def main():
    out = []
    for c in CASES:
        A = np.array(c["A"])
        At = np.ascontiguousarray(A.T)
        b = np.array(c["b"])
        x = C.brute_force(At, b, c["lam1"], c["lam2"])
        out.append(dict(c, x=[float(v) for v in x],
                        objective=float(C.primal_objective(At, b, x, c["lam1"], c["lam2"]))))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_en.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.checkers.brute_force (exhaustive sign enumeration)",
                   "cases": out}, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
