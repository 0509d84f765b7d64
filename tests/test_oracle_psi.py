"""Pins of the oracle's original Shan-Chen mode (Eq. 4-5): effective mass
psi = 1 - exp(-rho/rho0), force F = -G psi grad psi, pressure
p = rho c_s^2 + (G/2) psi^2.

Checked against what the mathematics fixes: the critical point of Eq. 5 in
closed form (rho_c = rho0 ln 2, G_c = -4 rho0 / 3), the identity of Eq. 4 with
the Eq. 22 form of the same potential U = (G/2) psi^2, the Zhang-Chen form on
smooth fields, exact conservation, fixed points, and the coexistence of a flat
interface: the force is an exact gradient in the continuum (psi grad psi =
grad psi^2 / 2), so the two phases settle at the equal-area pair of Eq. 5."""
import numpy as np
import pytest

import oracle


def psi(r, rho0=1.0):
    return 1.0 - np.exp(-r / rho0)


@pytest.mark.parametrize("rho0", [1.0, 0.5, 2.0])
def test_critical_point_closed_form(rho0):
    # d p/d rho = d^2 p/d rho^2 = 0 at rho_c = rho0 ln 2 when G = -4 rho0 / 3
    p = oracle.params_psi(4, 4, -4.0 * rho0 / 3.0, rho0=rho0)
    rc = rho0 * np.log(2.0)
    _, dp = oracle.p_eos(p, np.array([rc]))
    assert abs(dp[0]) < 1e-14
    h = 1e-4 * rho0
    _, dpp = oracle.p_eos(p, np.array([rc + h, rc - h]))
    assert abs((dpp[0] - dpp[1]) / (2 * h)) < 1e-8
    # above G_c there is no loop; below it there is
    with pytest.raises(Exception):
        oracle.maxwell(oracle.params_psi(4, 4, -1.2 * rho0, rho0=rho0))
    g, l, ps = oracle.maxwell(oracle.params_psi(4, 4, -2.0 * rho0, rho0=rho0))
    assert g < rc < l


def test_pressure_is_eq5():
    rho = np.linspace(0.05, 3.0, 41)
    for G in (-2.0, -3.5):
        pr, dp = oracle.p_eos(oracle.params_psi(4, 4, G), rho)
        assert np.allclose(pr, rho / 3 + 0.5 * G * psi(rho) ** 2, rtol=0, atol=1e-15)
        fd = (oracle.p_eos(oracle.params_psi(4, 4, G), rho + 1e-6)[0] -
              oracle.p_eos(oracle.params_psi(4, 4, G), rho - 1e-6)[0]) / 2e-6
        assert np.allclose(dp, fd, rtol=1e-8, atol=1e-10)


def field(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = 0.8 + 0.5 * np.sin(2 * np.pi * x / nx + rng.uniform(0, 6)) * np.cos(2 * np.pi * y / ny)
    return r + 0.05 * rng.standard_normal((ny, nx))


@pytest.mark.parametrize("grad", ["hdm", "cdm"])
def test_eq4_equals_eq22_form_of_the_same_potential(grad):
    # with U = (G/2) psi^2 (G < 0): Phi = sqrt|U| = sqrt(|G|/2) psi, s = sign U = -1,
    # so -2 s Phi D[Phi] = |G| psi D[psi] = -G psi D[psi] for any linear D
    nx, ny, G = 40, 36, -2.5
    r = field(nx, ny, 1)
    Fx, Fy = oracle.force(oracle.params_psi(nx, ny, G, grad=grad), r)
    phi = np.sqrt(abs(G) / 2) * psi(r)
    dx, dy = (oracle.hdm_grad if grad == "hdm" else oracle.cdm_grad)(phi)
    assert np.allclose(Fx, 2.0 * phi * dx, rtol=1e-12, atol=1e-14)
    assert np.allclose(Fy, 2.0 * phi * dy, rtol=1e-12, atol=1e-14)


def test_zc_form_agrees_on_smooth_fields():
    # -grad((G/2) psi^2) = -G psi grad psi in the continuum; the HDM keeps the
    # two discrete forms within its truncation error on a smooth field
    nx = ny = 128
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = 0.9 + 0.4 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    Fsc = oracle.force(oracle.params_psi(nx, ny, -2.0, force="sc"), r)
    Fzc = oracle.force(oracle.params_psi(nx, ny, -2.0, force="zc"), r)
    scale = np.abs(Fsc[0]).max()
    assert np.abs(Fsc[0] - Fzc[0]).max() < 1e-6 * scale
    assert np.abs(Fsc[1] - Fzc[1]).max() < 1e-6 * scale


@pytest.mark.parametrize("force", ["sc", "zc"])
def test_conservation_and_fixed_point(force):
    nx, ny = 32, 28
    p = oracle.params_psi(nx, ny, -1.5, force=force, tau=0.9)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = 0.8 + 0.2 * np.sin(2 * np.pi * x / nx) * np.cos(4 * np.pi * y / ny)
    f = oracle.init(p, r)
    m0 = f.sum()
    f = oracle.run(p, f, 20)
    assert f.sum() == pytest.approx(m0, rel=1e-13)
    jx = (oracle.EX[:, None, None] * f).sum()
    jy = (oracle.EY[:, None, None] * f).sum()
    assert abs(jx) < 1e-11 * m0 and abs(jy) < 1e-11 * m0     # the antisymmetric D conserves momentum
    u = oracle.init(p, np.full((ny, nx), 0.9))
    assert np.array_equal(oracle.step(p, u), u)


def test_flat_interface_coexistence_near_eq5_equal_area():
    # relaxed slab (G = -1.6, 10000 steps): bulk densities within 5 % of the
    # equal-area pair of Eq. 5 (they oscillate by ~2 % with the slow acoustic
    # mode of the periodic box), for both force forms
    nx, ny, G = 256, 4, -1.6
    for force in ("sc", "zc"):
        p = oracle.params_psi(nx, ny, G, force=force)
        g, l, _ = oracle.maxwell(p)
        x = np.arange(nx)
        r = g + 0.5 * (l - g) * (np.tanh(2 * (x - nx / 4) / 2.0) - np.tanh(2 * (x - 3 * nx / 4) / 2.0))
        f = oracle.run(p, oracle.init(p, np.tile(r, (ny, 1))), 10000)
        prof = f.sum(0).mean(0)
        liq = prof[nx // 2 - 8: nx // 2 + 9].mean()
        gas = np.r_[prof[:9], prof[-8:]].mean()
        assert abs(liq / l - 1) < 0.05 and abs(gas / g - 1) < 0.05, (force, liq, l, gas, g)
