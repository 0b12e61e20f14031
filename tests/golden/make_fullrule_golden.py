"""Write the oracle's full-rule solves stored in fullrule_<case>.json.

Each case is a seeded problem of the rectangular Gaussian family (x ~ N(0, I_2),
y ~ N((1,1), I_2/2), random marginals) at a reduced size, solved by the FP64
oracle (Algorithm 1, Sec. 3.1) from X_0 = p q^T until the
duality gap AND the l1 marginal residual are both <= 1e-6 (the stopping test of
Sec. 3.1 with the library's default quantities).  Every stored value comes from
``oracle.drot_solve`` only; the input hash (SHA-256 of the FP32 cost, then p and q
as FP64 bytes) lets the GPU test confirm that it solves the same problem.

A case takes minutes (384 x 512) to hours (768 x 1024) on one core; 1536 x 2048 would take
about ten hours there, so that case runs the oracle's OpenMP build (the same source: every
X_ij, r_i and s_j is formed as on one core, and only the three scalar totals - sum r, <C,X>,
r_dual^2 - are summed in another order).  Run from the repository root:
    python tests/golden/make_fullrule_golden.py <case> [<case> ...]
"""

import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

TOL = 1e-6
MAX_ITER = 4_000_000
CASES = {
    # name: (workload, seed, m, n, all host cores)
    "gauss_384x512": ("plain_8192x6144", 0, 384, 512, False),
    "gauss_768x1024": ("plain_8192x6144", 0, 768, 1024, False),
    "gauss_1536x2048": ("plain_8192x6144", 0, 1536, 2048, True),
}


def input_hash(C32, p, q) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(C32, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(p, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(q, dtype=np.float64).tobytes())
    return h.hexdigest()


def path_of(case: str) -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fullrule_{case}.json")


def main(names):
    for name in names:
        workload, seed, m, n, all_cores = CASES[name]
        pr = workloads.make_problem(workload, seed=seed, m=m, n=n)
        t0 = time.time()
        out = oracle.drot_solve(pr.C.astype(np.float64), pr.p, pr.q, pr.rho, tol=TOL, max_iter=MAX_ITER,
                                stop_rule=3, all_cores=all_cores)
        secs = time.time() - t0
        st = out["stats"]
        rec = dict(case=name, workload=workload, seed=seed, m=m, n=n, rho=pr.rho, tol=TOL, stop_rule="gap and l1",
                   input_sha256=input_hash(pr.C, pr.p, pr.q), status=out["status"], iters=out["iters"],
                   primal=st["primal"], dual=st["dual"], gap=st["gap"], res_l1=st["res_l1"], res_l2=st["res_l2"],
                   dual_res_prev=st["dual_res_prev"], oracle_threads=oracle.threads(all_cores),
                   oracle_seconds=round(secs, 1),
                   source=("oracle.drot_solve (FP64 C oracle, " + ("OpenMP build" if all_cores else "single thread")
                           + "), tests/golden/make_fullrule_golden.py"))
        with open(path_of(name), "w") as fh:
            json.dump(rec, fh, indent=1)
        print(f"{name}: status {out['status']} after {out['iters']} iterations, primal {st['primal']:.12g}, "
              f"{secs:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
