"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no step arithmetic of the method: it only draws initial
density fields and instance tables, on the host, in FP64.  Random numbers come
from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) keyed by (seed, cell index), so every consumer gets
identical inputs regardless of device or thread count.

Shapes follow the paper's workloads: a droplet in vapour (Sec. 5.4, spurious
currents), a flat liquid slab between vapour layers (Sec. 5.2, coexistence
curves) and a uniform mixture inside the spinodal with small noise (phase
separation).  Interfaces use the hyperbolic-tangent profile of Eq. 16.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20171216

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to uint64 counters ``x``."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of SplitMix64(seed ^ index)."""
    idx = np.arange(offset, offset + n, dtype=np.uint64) ^ np.uint64(seed)
    return (splitmix64(idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def droplet(nx: int, ny: int, radius: float, rho_g: float, rho_l: float,
            width: float = 2.0, cx: float | None = None, cy: float | None = None) -> np.ndarray:
    """Circular liquid droplet of radius ``radius`` centred at (cx, cy)
    (default: nx/2, ny/2), tanh interface of width ``width`` (Eq. 16 form).
    Returns a (ny, nx) float64 density field."""
    cx = nx / 2 if cx is None else cx
    cy = ny / 2 if cy is None else cy
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - radius) / width)


def splash(nx: int, ny: int, film: float, radius: float, speed: float, rho_g: float, rho_l: float,
           width: float = 4.0):
    """Droplet over a thin film (the splash case of Sec. 5.5): liquid below
    y = film along the bottom wall, a droplet of the given radius centred at
    x = nx/2 whose lowest point is four lattice spacings above the film, moving
    down at `speed`; tanh interfaces (Eq. 16 form).  Cell centres at i + 1/2
    (the walls lie at y = 0 and y = ny).  Returns (rho, ux, uy), (ny, nx) each."""
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    drop = 0.5 * (1 - np.tanh(2 * (np.hypot(X - nx / 2, Y - (film + 4 + radius)) - radius) / width))
    layer = 0.5 * (1 - np.tanh(2 * (Y - film) / width))
    rho = rho_g + (rho_l - rho_g) * np.clip(drop + layer, 0, 1)
    return rho, np.zeros_like(rho), -speed * drop


def slab(nx: int, ny: int, rho_g: float, rho_l: float, width: float = 2.0) -> np.ndarray:
    """Liquid in the middle half of x (interfaces at nx/4 and 3nx/4), vapour
    elsewhere, tanh interfaces (Eq. 16 form); uniform in y."""
    x = np.arange(nx, dtype=np.float64)
    x1, x2 = nx / 4.0, 3.0 * nx / 4.0
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (x - x1) / width)
                                            - np.tanh(2.0 * (x - x2) / width))
    return np.broadcast_to(prof, (ny, nx)).copy()


def spinodal(nx: int, ny: int, rho_mean: float, amp: float = 0.01,
             seed: int = DEFAULT_SEED) -> np.ndarray:
    """Uniform density with i.i.d. relative noise: rho_mean * (1 + amp (2 xi - 1)),
    xi = uniform01(seed, cell index)."""
    xi = uniform01(seed, nx * ny).reshape(ny, nx)
    return rho_mean * (1.0 + amp * (2.0 * xi - 1.0))


# Mean of the Carnahan-Starling (a=1, b=4, R=1) coexistence densities at
# T/Tc = 0.7 from the Maxwell construction: (0.009294146215 + 0.3581309412)/2.
# It lies inside the spinodal region, so a uniform state at this density
# separates into liquid and vapour.
CS_TR07_MEAN = 0.1837125437

# Equation-of-state constants of the sweeps (R = 1): VdW a=9/49 b=2/21 and
# CS a=1 b=4 as in Sec. 5.2; PR (omega = 0.344, water) and RK with a=2/49,
# b=2/21.  Hu scaling k as in Sec. 5.2: 0.01 VdW, 0.02 RK, 0.04 PR and CS.
EOS_TABLE = {
    "vdw": dict(a=9 / 49, b=2 / 21, omega=0.0, k=0.01),
    "cs": dict(a=1.0, b=4.0, omega=0.0, k=0.04),
    "pr": dict(a=2 / 49, b=2 / 21, omega=0.344, k=0.04),
    "rk": dict(a=2 / 49, b=2 / 21, omega=0.0, k=0.02),
}


def sweep_instances(n: int = 64, seed: int = DEFAULT_SEED, nx_lo: int = 256,
                    nx_hi: int = 2048, ny: int = 8, tr_lo: float = 0.5,
                    tr_hi: float = 0.95, tau_lo: float = 0.8, tau_hi: float = 1.2):
    """Instance table of the uneven temperature/EOS sweep: Nx drawn uniformly
    from the integers in [nx_lo, nx_hi], EOS drawn uniformly from EOS_TABLE,
    T/Tc evenly spaced over [tr_lo, tr_hi], tau uniform in [tau_lo, tau_hi].
    Each draw uses its own SplitMix64 stream."""
    names = sorted(EOS_TABLE)
    u_nx = uniform01(seed + 1, n)
    u_eos = uniform01(seed + 2, n)
    u_tau = uniform01(seed + 3, n)
    trs = np.linspace(tr_lo, tr_hi, n)
    out = []
    for i in range(n):
        nx = int(nx_lo + np.floor(u_nx[i] * (nx_hi - nx_lo + 1)))
        eos = names[int(np.floor(u_eos[i] * len(names)))]
        out.append(dict(nx=nx, ny=ny, eos=eos, Tr=float(trs[i]),
                        tau=float(tau_lo + (tau_hi - tau_lo) * u_tau[i]), **EOS_TABLE[eos]))
    return out
