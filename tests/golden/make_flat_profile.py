"""Writes flat_profile_vdw_tr09.txt: the equilibrium density profile across a
flat interface of the VdW fluid at T/Tc = 0.9 (Sec. 5.1, Eq. 24-26, Fig. 4),
computed by the FP64 oracle only (oracle.flat_profile).

VdW a = 9/49, b = 2/21 (the paper's VdW parameters), unscaled EOS (Sec. 5.1
uses no Hu factor); kappa = 0.05 (the paper does not give kappa: this value
makes the 10-90 % interface width 3.5 length units); grid spacing h = 0.5 as in
Fig. 4; 512 points, y = (i - 256) h, rising from rho_g to rho_l.

Usage: python tests/golden/make_flat_profile.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

A, B, TR, KAPPA, H, N = 9.0 / 49.0, 2.0 / 21.0, 0.9, 0.05, 0.5, 512
OUT = os.path.join(HERE, "flat_profile_vdw_tr09.txt")


def profile():
    p = oracle.params_at(1, 1, "vdw", A, B, TR)
    return oracle.flat_profile(p, KAPPA, H, N)


def main():
    y, rho, drho = profile()
    with open(OUT, "w") as fh:
        fh.write("# Equilibrium profile across a flat interface, VdW a=9/49 b=2/21 T/Tc=0.9 (Sec. 5.1,\n")
        fh.write("# Eq. 24-26 of arXiv:1712.06079), kappa=0.05, h=0.5; written by make_flat_profile.py\n")
        fh.write("# from the FP64 oracle.  Columns: y rho drho/dy\n")
        for a, b, c in zip(y, rho, drho):
            fh.write(f"{a:.1f} {b:.17g} {c:.17g}\n")


if __name__ == "__main__":
    main()
