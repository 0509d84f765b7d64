"""Laplace's law for a static droplet (Sec. 5.3, Table 1, Fig. 6) on the FP64
oracle: the pressure jump across the interface of a droplet of radius R is
Delta p = sigma / R in two dimensions, so Delta p against 1/R is a line
through the origin whose slope is the surface tension sigma.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  ``observables`` is the
measurement applied to a density field (the oracle's, or the CUDA path's in
the GPU tests, so both sides are read the same way); ``droplet_series`` runs
the oracle itself.

Readings (the paper gives neither the pressure tensor of the HDM model nor
how it measures the droplet): the pressure is the bulk p = k p_EOS of the
equation of state (Hu factor k of Sec. 5) inside and outside; the bulk
densities are the means of 5 x 5 cells at the droplet's centre and at the
lattice corner (the point farthest from the centre, periodic lattice); the
radius is the equivalent radius of the droplet's excess mass,
R = sqrt(sum_x (rho - rho_out) / (pi (rho_in - rho_out))).
"""
from __future__ import annotations

import numpy as np

from . import Params, init, moments, p_eos, run


def observables(p: Params, rho: np.ndarray):
    """(R_eq, rho_in, rho_out, Delta p) of a centred droplet field rho
    (shape (ny, nx), FP64 or FP32)."""
    r = np.asarray(rho, dtype=np.float64)
    ny, nx = r.shape
    rin = r[ny // 2 - 2: ny // 2 + 3, nx // 2 - 2: nx // 2 + 3].mean()
    rout = np.roll(np.roll(r, 2, 0), 2, 1)[:5, :5].mean()
    req = float(np.sqrt((r - rout).sum() / (np.pi * (rin - rout))))
    pe, _ = p_eos(p, np.array([rin, rout]))
    return req, float(rin), float(rout), float(p.k * (pe[0] - pe[1]))


def fit(points):
    """Least-squares Delta p = sigma / R + c over (R_eq, Delta p) pairs;
    returns (sigma, c, largest residual relative to the largest Delta p)."""
    x = np.array([1.0 / q[0] for q in points])
    y = np.array([q[1] for q in points])
    A = np.stack([x, np.ones_like(x)], axis=1)
    (sigma, c), *_ = np.linalg.lstsq(A, y, rcond=None)
    resid = y - (sigma * x + c)
    return float(sigma), float(c), float(np.abs(resid).max() / np.abs(y).max())


def droplet_series(p: Params, rho0s, steps: int):
    """Run the oracle from each initial density field (droplets made by the
    seeded input shapes) for `steps` steps and measure it; returns a list of
    (R_eq, rho_in, rho_out, Delta p)."""
    out = []
    for rho0 in rho0s:
        rho, _, _ = moments(p, run(p, init(p, rho0), steps))
        out.append(observables(p, rho))
    return out
