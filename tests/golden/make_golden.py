"""Write the exact optima stored in lp_optima.json.

Every value comes from the oracle package's exact solvers only (HiGHS LP via
``oracle.lp_optimum`` and, for uniform square problems, brute force over
permutations via ``oracle.permutation_optimum``) on inputs from the seeded
generators.  Run from the repository root:  python tests/golden/make_golden.py
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

CASES = [
    # (config, seed, m, n)
    ("plain_256", 0, 6, 6),
    ("plain_256", 1, 7, 7),
    ("plain_256", 2, 12, 9),
    ("plain_8192x6144", 0, 33, 31),
    ("warm_1024", 0, 40, 37),
    ("paper_gauss", 0, 48, 48),
    ("plain_20000", 0, 64, 61),
]


def main():
    out = []
    for name, seed, m, n in CASES:
        pr = workloads.make_problem(name, seed=seed, m=m, n=n)
        C = pr.C.astype(np.float64)
        opt, _ = oracle.lp_optimum(C, pr.p, pr.q)
        rec = dict(config=name, seed=seed, m=m, n=n, lp_optimum=opt, source="oracle.lp_optimum (HiGHS)")
        if m == n and m <= 7 and name == "plain_256":
            rec["permutation_optimum"] = oracle.permutation_optimum(C)
        out.append(rec)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lp_optima.json")
    with open(path, "w") as fh:
        json.dump(dict(note="Exact OT optima of seeded workloads (eq. ot:dist), written by make_golden.py",
                       cases=out), fh, indent=1)
    print(f"wrote {len(out)} cases to {path}")


if __name__ == "__main__":
    main()
