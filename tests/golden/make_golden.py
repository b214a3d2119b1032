"""Write the stored expected values of tests/golden/ from the oracle alone.

small_k.json: the n = 2,048 stand-in for the paper's smallest workload (periodic diamond 4x4x4
cells, seed 0, gen.workload("small"), k = n/2 as for the half-filled band of Appendix B):
lambda_{k-2} .. lambda_{k+2} from the oracle's dense generalized eigensolver (c2, Cholesky
reduction as in the dense comparison solver of Section 4.2) and nu_sigma(A, B) at certified
shifts from the oracle's dense Bunch-Kaufman inertia (c1; Sylvester's law, Section 2.1).  These
are not values printed in the paper: its k-th eigenvalues are for ELSES matrices that are not
available here.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from gen import workload          # noqa: E402
from oracle import core           # noqa: E402


def main():
    p = workload("small", seed=0)
    A, B = p.A().toarray(), p.B().toarray()
    lam, _ = core.gen_eig(A, B)
    k = p.k
    nrm = float(np.abs(A).sum(1).max())
    shifts = core.certified_shifts(lam, 6, 1e-8 * nrm, seed=31)
    nus = [core.dense_nu(A, B, float(s)) for s in shifts]
    out = {
        "workload": "small (periodic diamond 4x4x4 cells, seed 0)",
        "source": "oracle (c2) dense generalized eigensolver and (c1) dense Bunch-Kaufman inertia",
        "n": p.n, "k": k, "norm_a_inf": nrm,
        "lambda": {str(i): float(lam[i - 1]) for i in range(k - 2, k + 3)},
        "shifts": [float(s) for s in shifts], "nu": nus,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_k.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
