"""Write tests/golden/oracle_elements.json from the oracle alone.

Inputs come from the seeded generator; outputs are the oracle's FP64 element
matrices and load vectors for p = 1 and 2 on the first 4 elements of a
+-25% jitter mesh.  The file pins the oracle across machines (the same C
source compiled on x86 and on aarch64 must give the same values).
Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1310_1194_gb300 import inputs  # noqa: E402


def main():
    n = 4
    geom = inputs.prism_mesh(4, 4, 2, 0.25, seed=7)[:n]
    coef = inputs.coefficients(n, seed=7)
    out = {"source": "oracle/fei_oracle.c via tests/golden/make_golden.py",
           "geom": geom.tolist(), **{k: v.tolist() for k, v in coef.items()}}
    for p in (1, 2):
        A, bv, st, _ = oracle.integrate(geom, coef["K"], coef["b"], coef["c"], coef["f"], p=p)
        assert not st.any()
        out[f"A_p{p}"] = [repr(float(x)) for x in A]
        out[f"b_p{p}"] = [repr(float(x)) for x in bv]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_elements.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
