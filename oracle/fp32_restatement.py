"""The oracle's time step restated in numpy with a chosen arithmetic and
storage precision, to measure what FP32 can reach.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests import it;
the product library never does.  It shares no code with the CUDA path.

The step is the oracle's (``lbm_oracle.c``, ``step_with``), operation by
operation and in the same order, on whole fields:
  rho = sum_i f_i, j = sum_i e_i f_i, u = j / rho                     (Eq. 3)
  U = k p_EOS(rho, T) - rho/3 (Eq. 8, Hu factor of Sec. 5; EOS Eq. 24, 27-29)
  Shan-Chen: Phi = sqrt|U| (Eq. 21), F = -2 s Phi D[Phi], s = sign U  (Eq. 22)
  Zhang-Chen: F = -D[U]                                                (Eq. 7)
  f_i* = f_i - (f_i - f^eq_i(rho, u))/tau
         + [f^eq_i(rho, u + F/rho) - f^eq_i(rho, u)]             (Eq. 1, 2, 10)
  f_i(x + e_i, t + 1) = f_i*(x), periodic.
D is the periodic HDM operator of Eq. 20 along rows and columns, or with
``grad == "cdm"`` the weighted central difference of Eq. 15 normalised by
1/c_s^2 = 3 (D_x = 3 sum_i w_i q(x + e_i) e_ix, the eight neighbours).  The HDM's explicit
form, d_i = sum_j w_j (q_(i+j) - q_(i-j)), takes its weights from the oracle's
own cyclic solve (the response of ``oracle.hdm_line`` to a unit impulse), over
the whole period, so with FP64 arithmetic this restatement is the oracle's
operator to rounding.  The sum runs from the farthest pair to the nearest.

``arith`` is the precision of every operation (``np.float32`` or
``np.float64``); ``store`` the precision the nine distributions are kept in
between steps.  FP64 arithmetic with FP32 storage rounds only the stored state;
FP32 arithmetic rounds every operation as a plain FP32 evaluation would.
"""
from __future__ import annotations

import numpy as np

from . import Params, hdm_line

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def periodic_weights(n: int) -> np.ndarray:
    """w_1 .. w_K of the explicit periodic HDM operator on n points: the
    oracle's solve of Eq. 20 applied to a unit impulse at 0 gives d_(-j) = w_j.
    K is half the period, or less where the weights (which fall off as
    0.382^j) drop below 1e-18 of w_1, where they change no FP64 sum."""
    imp = np.zeros(n)
    imp[0] = 1.0
    d = hdm_line(imp)
    w = np.array([d[n - j] for j in range(1, n // 2 + 1)])
    keep = np.nonzero(np.abs(w) > 1e-18 * abs(w[0]))[0]
    return w[: keep[-1] + 1]


def _alpha(p: Params) -> float:
    if p.eos == "pr":       # Eq. 28
        m = 0.37464 + 1.54226 * p.omega - 0.26992 * p.omega ** 2
        return (1.0 + m * (1.0 - np.sqrt(p.T / p.Tc))) ** 2
    if p.eos == "rks":      # the Soave form after Eq. 27
        m = 0.480 + 1.574 * p.omega - 0.176 * p.omega ** 2
        return (1.0 + m * (1.0 - np.sqrt(p.T / p.Tc))) ** 2
    if p.eos == "rk":       # Eq. 27
        return 1.0 / np.sqrt(p.T)
    return 1.0


class Restatement:
    """The step of ``p`` (periodic, HDM, an equation of state) in the given
    arithmetic and storage precision."""

    def __init__(self, p: Params, arith=np.float32, store=np.float32):
        if p.walls or p.grad not in ("hdm", "cdm") or p.eos == "psi":
            raise ValueError("the restatement covers the periodic step with an equation of state")
        self.p, self.t, self.store = p, arith, store
        t = arith
        self.wx = [t(w) for w in periodic_weights(p.nx)]
        self.wy = [t(w) for w in periodic_weights(p.ny)]
        self.c = dict(a=t(p.a), b=t(p.b), RT=t(p.R * p.T), aal=t(p.a * _alpha(p)), k=t(p.k),
                      third=t(1) / t(3), tau=t(p.tau), w=[t(w) for w in W9])

    def _D(self, q, w, axis):
        if self.p.grad == "cdm":   # Eq. 15: 3 (w_axis (q_+ - q_-) + w_diag ((q_++ + q_+-) - (q_-+ + q_--)))
            t, other = self.t, 1 - axis
            up, dn = np.roll(q, -1, axis), np.roll(q, 1, axis)
            diag = (np.roll(up, -1, other) + np.roll(up, 1, other)) - (np.roll(dn, -1, other) + np.roll(dn, 1, other))
            return t(3) * (t(1 / 9) * (up - dn) + t(1 / 36) * diag)
        out = np.zeros_like(q)
        for j in range(len(w), 0, -1):
            out = out + w[j - 1] * (np.roll(q, -j, axis) - np.roll(q, j, axis))
        return out

    def _p_eos(self, rho):
        t, c, eos = self.t, self.c, self.p.eos
        if eos == "cs":     # Eq. 29 with the standard (1 - b rho/4)^3
            e = c["b"] * rho / t(4)
            om = t(1) - e
            return rho * c["RT"] * (t(1) + e + e * e - e * e * e) / (om * om * om) - c["a"] * rho * rho
        rep = rho * c["RT"] / (t(1) - c["b"] * rho)
        if eos == "vdw":    # Eq. 24
            return rep - c["a"] * rho * rho
        if eos == "pr":     # Eq. 28
            return rep - c["aal"] * rho * rho / (t(1) + t(2) * c["b"] * rho - c["b"] * c["b"] * rho * rho)
        return rep - c["aal"] * rho * rho / (t(1) + c["b"] * rho)   # RK, RKS (Eq. 27)

    def _feq(self, i, rho, ux, uy):
        t = self.t
        eu = t(EX[i]) * ux + t(EY[i]) * uy
        uu = ux * ux + uy * uy
        return rho * self.c["w"][i] * (t(1) + t(3) * eu + t(4.5) * eu * eu - t(1.5) * uu)

    def step(self, f: np.ndarray) -> np.ndarray:
        """One step of a (9, ny, nx) state kept in the storage precision."""
        t, c = self.t, self.c
        f = f.astype(t)
        rho = f[0].copy()
        jx = t(EX[0]) * f[0]
        jy = t(EY[0]) * f[0]
        for i in range(1, 9):
            rho = rho + f[i]
            jx = jx + t(EX[i]) * f[i]
            jy = jy + t(EY[i]) * f[i]
        ux, uy = jx / rho, jy / rho
        U = c["k"] * self._p_eos(rho) - rho * c["third"]
        if self.p.force == "sc":
            fld = np.sqrt(np.abs(U))
            s = np.where(U >= t(0), t(1), t(-1))
            Fx = t(-2) * s * fld * self._D(fld, self.wx, 1)
            Fy = t(-2) * s * fld * self._D(fld, self.wy, 0)
        else:
            Fx = -self._D(U, self.wx, 1)
            Fy = -self._D(U, self.wy, 0)
        vx, vy = ux + Fx / rho, uy + Fy / rho
        out = np.empty(f.shape, dtype=self.store)
        for i in range(9):
            fe = self._feq(i, rho, ux, uy)
            fs = self._feq(i, rho, vx, vy)
            post = f[i] - (f[i] - fe) / c["tau"] + (fs - fe)
            out[i] = np.roll(np.roll(post, EX[i], 1), EY[i], 0)
        return out

    def run(self, f0: np.ndarray, nsteps: int) -> np.ndarray:
        """nsteps steps from the FP64 state f0 (rounded to the storage
        precision first); returns the state as FP64."""
        f = np.asarray(f0, dtype=np.float64).astype(self.store)
        for _ in range(nsteps):
            f = self.step(f)
        return f.astype(np.float64)
