"""Writes laplace_vdw_oracle.txt: Laplace's law (Sec. 5.3) on the FP64 oracle.
VdW droplets (a = 9/49, b = 2/21, R = 1, Hu factor k = 0.01 of Sec. 5.2,
tau = 1, Shan-Chen force with the HDM gradient) on periodic lattices:
T/Tc = 0.6 on 96 x 96 with initial radii 15, 20, 25 after 5000 steps, and
T/Tc = 0.8 on 128 x 128 with radii 25, 30, 35 after 8000 steps (the wider
interface at 0.8 needs larger droplets).  Each droplet starts from the seeded
input shape (Maxwell densities, tanh interface of width 2, centred) and is
measured by oracle.laplace.observables.  Calls only oracle/ (and the seeded
input shapes).

Usage: python tests/golden/make_laplace_oracle.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import laplace  # noqa: E402
from paper_1712_06079_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "laplace_vdw_oracle.txt")
# (T/Tc, lattice side, steps, initial radii)
SERIES = [(0.6, 96, 5000, (15, 20, 25)), (0.8, 128, 8000, (25, 30, 35))]


def params(Tr, n):
    t = inputs.EOS_TABLE["vdw"]
    return oracle.params_at(n, n, "vdw", t["a"], t["b"], Tr, k=t["k"], tau=1.0, force="sc", grad="hdm")


def initial(p, R0):
    g, l, _ = oracle.maxwell(p)
    return inputs.droplet(p.nx, p.ny, R0, g, l)


def series():
    rows = []
    for Tr, n, steps, radii in SERIES:
        p = params(Tr, n)
        obs = laplace.droplet_series(p, [initial(p, R0) for R0 in radii], steps)
        rows += [(Tr, n, steps, R0) + o for R0, o in zip(radii, obs)]
    return rows


def main():
    oracle.set_threads(oracle.max_threads())
    with open(OUT, "w") as fh:
        fh.write("# Laplace's law on the FP64 oracle (Sec. 5.3): VdW a=9/49 b=2/21 k=0.01 tau=1, SC + HDM,\n")
        fh.write("# droplets measured by oracle.laplace.observables; written by make_laplace_oracle.py.\n")
        fh.write("# Columns: Tr n steps R0 R_eq rho_in rho_out dp\n")
        for Tr, n, steps, R0, req, rin, rout, dp in series():
            fh.write(f"{Tr} {n} {steps} {R0} {req:.15g} {rin:.15g} {rout:.15g} {dp:.15g}\n")


if __name__ == "__main__":
    main()
