"""Write tests/golden/oracle_outer_its.txt: outer FGMRES iterations the CPU oracle
needs on the benchmark workloads (calls oracle/ and the seeded input generator only).

Run from the repository root:  python tests/golden/make_oracle_counts.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solve  # noqa: E402
from paper_2506_03947_gb300 import inputs  # noqa: E402

CASES = [
    ("2d_lognormal_1024x1024_l10_a1e-2_p40", lambda: inputs.config_2d_large(inner_its=40)),
    ("2d_lognormal_1024x1024_l10_a1e-2_p10", lambda: inputs.config_2d_large(inner_its=10)),
    ("2d_lognormal_256x256_l10_a1e-2_p20", lambda: inputs.config_2d(alpha=1e-2)),
]


def main():
    out = os.path.join(ROOT, "tests", "golden", "oracle_outer_its.txt")
    lines = ["# Outer FGMRES iterations of the CPU oracle (MGS, x_0 = 0) to explicit",
             "# relative residual 1e-8; written by tests/golden/make_oracle_counts.py.",
             "# Columns: workload, outer_its, explicit_residual, oracle_seconds"]
    for name, mk in CASES:
        P = mk()
        t = time.time()
        r = solve.solve(P.kx, P.ky, P.kz, P.shape, P.ell, P.alpha, P.b, P.inner_its, 1e-8, 64)
        dt = time.time() - t
        assert r.converged
        lines.append("%s %d %.3e %.1f" % (name, r.outer_its, r.resid_explicit, dt))
        print(lines[-1], flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
