"""Writes fp32_restatement_errors.txt: the pointwise density error after 1000
steps, max_x |rho - rho64| / |rho64|, of the oracle's step restated in numpy
(oracle/fp32_restatement.py) with FP32 storage and FP32 or FP64 arithmetic,
against the FP64 oracle, on the two FP32 parity workloads: the 128^2 CS
droplet (T/Tc 0.8, R 30, Shan-Chen, HDM) and the 1024 x 8 PR slab (T/Tc 0.7,
Zhang-Chen, HDM), tau = 1, Hu factor k = 0.04.  Calls only oracle/ (and the
seeded input shapes).

Usage: python tests/golden/make_fp32_limits.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle.fp32_restatement import Restatement  # noqa: E402
from paper_1712_06079_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "fp32_restatement_errors.txt")


def workload(case):
    if case == "droplet":
        t = inputs.EOS_TABLE["cs"]
        op = oracle.params_at(128, 128, "cs", t["a"], t["b"], 0.8, k=t["k"], force="sc")
        g, l, _ = oracle.maxwell(op)
        return op, inputs.droplet(128, 128, 30, g, l)
    t = inputs.EOS_TABLE["pr"]
    op = oracle.params_at(1024, 8, "pr", t["a"], t["b"], 0.7, omega=t["omega"], k=t["k"], force="zc")
    g, l, _ = oracle.maxwell(op)
    return op, inputs.slab(1024, 8, g, l)


def main():
    rows = []
    for case in ("droplet", "slab"):
        op, rho0 = workload(case)
        f0 = oracle.init(op, rho0)
        ro = oracle.run(op, f0, 1000).sum(0)
        for arith, name in ((np.float32, "f32"), (np.float64, "f64")):
            r = Restatement(op, arith, np.float32).run(f0, 1000).sum(0)
            rows.append((case, name, "f32", float(np.max(np.abs(r - ro) / np.abs(ro)))))
    with open(OUT, "w") as fh:
        fh.write("# Pointwise rho error after 1000 steps, max_x |rho - rho64| / |rho64|, of the oracle's step\n")
        fh.write("# restated with the given arithmetic and storage precision (oracle/fp32_restatement.py),\n")
        fh.write("# against the FP64 oracle; written by make_fp32_limits.py.  Columns: case arith store error\n")
        for case, arith, store, err in rows:
            fh.write(f"{case} {arith} {store} {err:.9e}\n")


if __name__ == "__main__":
    main()
