"""Pins of the oracle's equations of state, critical points and Maxwell
construction (Sec. 5.2, Eq. 24, 27-29) against closed forms and textbook
constants -- nothing here re-types the oracle's own formulas."""
import math

import numpy as np
import pytest

import oracle

VDW = dict(a=9 / 49, b=2 / 21)
CS = dict(a=1.0, b=4.0)
PR = dict(a=2 / 49, b=2 / 21)
RK = dict(a=2 / 49, b=2 / 21)


def test_vdw_critical_point_closed_form():
    # Eq. 24: Tc = 8a/(27 b R), rho_c = 1/(3b)  (4/7 and 3.5 for the paper's a, b)
    Tc, rc = oracle.critical_point("vdw", **VDW)
    assert Tc == pytest.approx(8 * VDW["a"] / (27 * VDW["b"]), rel=1e-14)
    assert Tc == pytest.approx(4 / 7, rel=1e-14)
    assert rc == pytest.approx(1 / (3 * VDW["b"]), rel=1e-7)
    # critical pressure 3/8 R Tc rho_c ... p_c = a/(27 b^2)
    p = oracle.Params(1, 1, "vdw", T=Tc, **VDW)
    pc, dpc = oracle.p_eos(p, np.array([1 / (3 * VDW["b"])]))
    assert pc[0] == pytest.approx(VDW["a"] / (27 * VDW["b"] ** 2), rel=1e-12)
    assert abs(dpc[0]) < 1e-12


@pytest.mark.parametrize("a,b", [(1.0, 4.0), (0.5, 2.0), (2.0, 1.0)])
def test_cs_critical_point_textbook(a, b):
    # Carnahan-Starling repulsion with vdW attraction: a = 0.4963 R^2 Tc^2/pc,
    # b = 0.18727 R Tc/pc (Yuan & Schaefer 2006), critical packing fraction
    # eta_c = b rho_c / 4 = 0.13044.  Four-digit literature constants.
    Tc, rc = oracle.critical_point("cs", a, b)
    assert Tc == pytest.approx(0.18727 / 0.4963 * a / b, rel=3e-4)
    assert b * rc / 4 == pytest.approx(0.13044, rel=3e-4)


def test_pr_critical_point_textbook():
    # Peng & Robinson (1976): a = 0.45724 R^2 Tc^2/pc, b = 0.07780 R Tc/pc, Zc = 0.3074
    Tc, rc = oracle.critical_point("pr", **PR)
    assert Tc == pytest.approx(0.07780 / 0.45724 * PR["a"] / PR["b"], rel=3e-4)
    assert rc == pytest.approx(0.07780 / (PR["b"] * 0.3074), rel=5e-4)


def test_rk_critical_point_textbook():
    # Redlich & Kwong (1949): a = 0.42748 R^2 Tc^2.5/pc, b = 0.08664 R Tc/pc, Zc = 1/3
    Tc, rc = oracle.critical_point("rk", **RK)
    assert Tc ** 1.5 == pytest.approx(0.08664 / 0.42748 * RK["a"] / RK["b"], rel=3e-4)
    assert rc == pytest.approx(0.08664 * 3 / RK["b"], rel=5e-4)


def test_rks_critical_point_matches_rk_with_alpha_one():
    # RKS with alpha(Tc) = 1 has the critical density of RK and Tc^1 scaling
    Tc, rc = oracle.critical_point("rks", **VDW)
    assert Tc == pytest.approx(0.08664 / 0.42748 * VDW["a"] / VDW["b"], rel=3e-4)
    assert rc == pytest.approx(0.08664 * 3 / VDW["b"], rel=5e-4)


def test_cs_virial_expansion():
    # The Carnahan-Starling compressibility factor reproduces the hard-sphere
    # virial series Z = 1 + 4 eta + 10 eta^2 + 18 eta^3 + 28 eta^4 + 40 eta^5 ...
    # (coefficients n^2 + n - 2).  With a = 0 the EOS is p = rho R T Z(eta),
    # eta = b rho / 4; the printed denominator (1 - eta^3) of Eq. 29 would fail.
    p = oracle.Params(1, 1, "cs", a=0.0, b=4.0, T=1.0)
    eta = np.array([1e-3, 3e-3, 1e-2])
    rho = 4 * eta / p.b
    pv, _ = oracle.p_eos(p, rho)
    Z = pv / rho
    series = 1 + 4 * eta + 10 * eta ** 2 + 18 * eta ** 3 + 28 * eta ** 4 + 40 * eta ** 5
    assert np.allclose(Z, series, rtol=0, atol=60 * eta ** 6 + 1e-14)


@pytest.mark.parametrize("eos,pars", [("vdw", VDW), ("cs", CS), ("pr", PR), ("rk", RK), ("rks", VDW)])
def test_ideal_gas_limit_and_derivative(eos, pars):
    p = oracle.params_at(1, 1, eos, pars["a"], pars["b"], 0.8, omega=0.344)
    rho = np.array([1e-9])
    pv, dp = oracle.p_eos(p, rho)
    assert pv[0] / rho[0] == pytest.approx(p.T, rel=1e-6)  # p -> rho R T
    # analytic dp/drho against a central difference of p
    pole = 4 / pars["b"] if eos == "cs" else 1 / pars["b"]
    r = np.linspace(0.02, 0.9, 23) * pole
    h = 1e-6 * pole
    pp, _ = oracle.p_eos(p, r + h)
    pm, _ = oracle.p_eos(p, r - h)
    _, d = oracle.p_eos(p, r)
    scale = np.abs(pp).max() / pole
    assert np.allclose(d, (pp - pm) / (2 * h), rtol=1e-6, atol=1e-6 * scale)


def test_pr_alpha_is_one_at_tc():
    # alpha(T) of Eq. 28 equals 1 at Tr = 1, so (Tc, rho_c) of the alpha = 1
    # form is the critical point of the full PR EOS: dp/drho = 0 there and
    # negative just below Tc.
    Tc, rc = oracle.critical_point("pr", **PR)
    p = oracle.Params(1, 1, "pr", omega=0.344, T=Tc, Tc=Tc, **PR)
    _, d = oracle.p_eos(p, np.array([0.5 * rc, rc]))
    assert abs(d[1]) < 1e-7 * d[0]
    p.T = 0.99 * Tc
    _, d = oracle.p_eos(p, np.array([rc]))
    assert d[0] < 0


# --- Maxwell construction -------------------------------------------------

def mu_vdw(rho, T, a, b):
    # chemical potential of the VdW fluid (up to a T-only constant):
    # mu = T ln(rho/(1 - b rho)) + T/(1 - b rho) - 2 a rho;  p = rho mu - f
    return T * np.log(rho / (1 - b * rho)) + T / (1 - b * rho) - 2 * a * rho


def mu_cs(rho, T, a, b):
    # CS excess free energy per particle (4 eta - 3 eta^2)/(1 - eta)^2;
    # mu = T[ln rho + (4e - 3e^2)/(1-e)^2 + e (4 - 2e)/(1-e)^3] - 2 a rho
    e = b * rho / 4
    return T * (np.log(rho) + (4 * e - 3 * e * e) / (1 - e) ** 2 + e * (4 - 2 * e) / (1 - e) ** 3) - 2 * a * rho


def mu_rk(rho, T, a, b):
    # RK (Eq. 27) with alpha = 1/sqrt(T):
    # mu = T ln(rho/(1-b rho)) + T/(1-b rho) - (a alpha/b)[ln(1+b rho) + b rho/(1+b rho)]
    al = 1 / math.sqrt(T)
    return (T * np.log(rho / (1 - b * rho)) + T / (1 - b * rho)
            - a * al / b * (np.log(1 + b * rho) + b * rho / (1 + b * rho)))


@pytest.mark.parametrize("eos,pars,mu", [("vdw", VDW, mu_vdw), ("cs", CS, mu_cs), ("rk", RK, mu_rk)])
@pytest.mark.parametrize("Tr", [0.5, 0.7, 0.9, 0.98])
def test_maxwell_equal_chemical_potential(eos, pars, mu, Tr):
    # Equal areas <=> equal pressure and equal chemical potential (closed-form mu)
    p = oracle.params_at(1, 1, eos, pars["a"], pars["b"], Tr)
    g, l, ps = oracle.maxwell(p)
    assert g < l
    pv, _ = oracle.p_eos(p, np.array([g, l]))
    assert pv[0] == pytest.approx(ps, rel=1e-10)
    assert pv[1] == pytest.approx(ps, rel=1e-10)
    mg, ml = mu(np.array([g, l]), p.T, pars["a"], pars["b"])
    assert abs(mg - ml) < 1e-9 * (abs(mg) + p.T)


def test_maxwell_near_critical_scaling():
    # VdW near Tc: (rho_l - rho_g)/rho_c -> 4 sqrt(1 - Tr)
    for Tr in (0.9999, 0.99999):
        p = oracle.params_at(1, 1, "vdw", VDW["a"], VDW["b"], Tr)
        g, l, _ = oracle.maxwell(p)
        rc = 1 / (3 * VDW["b"])
        assert (l - g) / rc == pytest.approx(4 * math.sqrt(1 - Tr), rel=2 * (1 - Tr) ** 0.5 + 1e-4)


def test_maxwell_corresponding_states():
    # VdW coexistence in units of rho_c depends on Tr only (any a, b)
    out = []
    for a, b in [(9 / 49, 2 / 21), (1.0, 1.0), (0.3, 0.05)]:
        p = oracle.params_at(1, 1, "vdw", a, b, 0.6)
        g, l, _ = oracle.maxwell(p)
        out.append((g * 3 * b, l * 3 * b))
    for o in out[1:]:
        assert o == pytest.approx(out[0], rel=1e-9)


def test_maxwell_no_loop_above_tc():
    p = oracle.params_at(1, 1, "vdw", VDW["a"], VDW["b"], 1.05)
    with pytest.raises(RuntimeError):
        oracle.maxwell(p)


def test_cs_tr07_mean_input_constant():
    # the spinodal workload's mean density is the mean of the CS Tr=0.7 coexistence pair
    from paper_1712_06079_gb300 import inputs
    p = oracle.params_at(1, 1, "cs", 1.0, 4.0, 0.7)
    g, l, _ = oracle.maxwell(p)
    assert 0.5 * (g + l) == pytest.approx(inputs.CS_TR07_MEAN, rel=1e-9)
    # and it lies inside the spinodal (dp/drho < 0): a uniform state there is unstable
    _, d = oracle.p_eos(p, np.array([inputs.CS_TR07_MEAN]))
    assert d[0] < 0
