"""Pins of the oracle's flat-interface equilibrium profile (Sec. 5.1, Eq. 25-26,
Fig. 4) and of the golden profile written from it.

The oracle integrates the first integral (kappa/2) rho'^2 = W(rho) of Eq. 26.
The pins check the equation itself, not the first integral: the bracket
p - kappa rho rho'' + (kappa/2) rho'^2 of Eq. 25-26, with rho'' and rho' by
eighth-order differences of the sampled profile, equals the Maxwell
coexistence pressure everywhere; the returned slope equals the difference
quotient; the profile joins the two Maxwell densities; the width scales as
sqrt(kappa); and on the exact profile the HDM derivative (Eq. 20) is far closer
to the exact slope than the CDM one (Eq. 15), the claim of Fig. 4."""
import os
import runpy

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
C1 = np.array([1 / 280, -4 / 105, 1 / 5, -4 / 5, 0, 4 / 5, -1 / 5, 4 / 105, -1 / 280])
C2 = np.array([-1 / 560, 8 / 315, -1 / 5, 8 / 5, -205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560])


def central(r, c, h, order):
    i = np.arange(4, len(r) - 4)
    return i, sum(c[k] * r[i + k - 4] for k in range(9)) / h ** order


@pytest.mark.parametrize("eos,a,b,tr,kappa", [("vdw", 9 / 49, 2 / 21, 0.9, 0.05), ("vdw", 9 / 49, 2 / 21, 0.7, 0.2),
                                             ("cs", 1.0, 4.0, 0.8, 0.5), ("pr", 2 / 49, 2 / 21, 0.75, 0.1)])
def test_profile_satisfies_eq26(eos, a, b, tr, kappa):
    p = oracle.params_at(1, 1, eos, a, b, tr)
    g, l, ps = oracle.maxwell(p)
    h = 1 / 32
    y, r, d = oracle.flat_profile(p, kappa, h, 32 * 100 + 1, sub=16)   # y in [-50, 50]
    i, d1 = central(r, C1, h, 1)
    _, d2 = central(r, C2, h, 2)
    pe, _ = oracle.p_eos(p, r[i])
    bracket = pe - kappa * r[i] * d2 + 0.5 * kappa * d1 ** 2
    # the floor is rounding in the second difference, ~ kappa rho eps / h^2
    assert np.abs(bracket - ps).max() < 5e-9 * ps
    assert np.abs(d1 - d[i]).max() < 1e-9 * d.max()
    assert np.all(np.diff(r) > 0) or np.all(np.diff(r) >= 0)
    assert abs(r[0] - g) < 1e-9 * g and abs(r[-1] - l) < 1e-9 * l
    assert np.all(r > g - 1e-12) and np.all(r < l + 1e-12)
    # y = 0 at the mean density
    assert r[len(r) // 2] == pytest.approx(0.5 * (g + l), rel=1e-12)


def test_profile_width_scales_with_sqrt_kappa():
    # rho' = sqrt(2 W / kappa): the profile at 4 kappa is the profile at kappa stretched by 2
    p = oracle.params_at(1, 1, "vdw", 9 / 49, 2 / 21, 0.9)
    _, r1, d1 = oracle.flat_profile(p, 0.05, 0.25, 201)
    _, r4, d4 = oracle.flat_profile(p, 0.20, 0.50, 201)
    assert np.abs(r1 - r4).max() < 1e-11
    assert np.abs(d1 - 2 * d4).max() < 1e-10


def test_profile_rejects_bad_arguments():
    p = oracle.params_at(1, 1, "vdw", 9 / 49, 2 / 21, 0.9)
    for kappa, h, n in ((0.0, 0.5, 10), (0.05, -1.0, 10), (0.05, 0.5, 0)):
        with pytest.raises(RuntimeError):
            oracle.flat_profile(p, kappa, h, n, i0=0)
    with pytest.raises(RuntimeError):   # above the critical temperature: no two-phase profile
        oracle.flat_profile(oracle.params_at(1, 1, "vdw", 9 / 49, 2 / 21, 1.05), 0.05, 0.5, 10)


def load_golden():
    rows = np.loadtxt(os.path.join(HERE, "golden", "flat_profile_vdw_tr09.txt"))
    return rows[:, 0], rows[:, 1], rows[:, 2]


def test_golden_profile_is_the_oracles():
    # the stored fixture is exactly what its committed script writes from the oracle
    mod = runpy.run_path(os.path.join(HERE, "golden", "make_flat_profile.py"))
    y, r, d = mod["profile"]()
    gy, gr, gd = load_golden()
    assert np.array_equal(gy, y)
    assert np.abs(gr - r).max() <= 4e-16 * r.max()
    assert np.abs(gd - d).max() <= 4e-16 * d.max()


def test_fig4_hdm_closer_than_cdm_on_exact_profile():
    # Fig. 4 (h = 0.5): on the real equilibrium profile HDM is far closer to the
    # exact slope than CDM.  The line is made periodic by its mirror image (two
    # interfaces 256 length units apart; the tails are at bulk to rounding).
    y, r, d = load_golden()
    h = 0.5
    line = np.concatenate([r, r[::-1]])
    exact = np.concatenate([d, -d[::-1]])
    hdm = oracle.hdm_line(line) / h
    cdm = oracle.cdm_grad(np.tile(line[:, None], (1, 3)))[1][:, 1] / h
    e_h = np.abs(hdm - exact).max() / np.abs(exact).max()
    e_c = np.abs(cdm - exact).max() / np.abs(exact).max()
    assert e_h < 2e-4
    assert e_c > 1e-2
    assert e_c > 100 * e_h
    # the profile is not a tanh: its slope is not symmetric about y = 0
    i0 = len(y) // 2
    assert abs(d[i0 - 1] - d[i0 + 1]) > 1e-2 * d[i0]
