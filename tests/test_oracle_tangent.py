"""Pins of the oracle's complex-step derivative of the discrete map.

The step is run in complex arithmetic with imaginary parts i h on the
temperature, G or the initial density (Squire & Trapp 1998).  The imaginary
part of the final density over h is then the derivative, with no difference
quotient.  Checked here against constructions other than itself:
- the real part is the real oracle run;
- Richardson-extrapolated central differences of the real oracle, for every
  equation of state, both force forms, both gradients, tau != 1, walls, and
  the G of the original effective mass (Eq. 4);
- in the sign-mixing regime of Eq. 22 (U > 0 in some cells), central
  differences converge to it as h^2;
- mass conservation of the tangent map (sum of d rho_T = sum of d rho_0);
- linearity in the direction;
- a uniform state has zero temperature derivative (no force for any T)."""
import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs

EOS = dict(inputs.EOS_TABLE)
EOS["rks"] = dict(a=9 / 49, b=2 / 21, omega=0.344, k=0.01)


def params(eos, Tr, force="sc", grad="hdm", tau=1.0, walls=False, nx=24, ny=20, k=None):
    t = EOS[eos]
    return oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=t["k"] if k is None else k,
                            tau=tau, force=force, grad=grad, walls=walls)


def droplet(op, R=5.0):
    g, l, _ = oracle.maxwell(op)
    return inputs.droplet(op.nx, op.ny, R, g, l), l - g


def final_rho(op, rho0, n):
    return oracle.run(op, oracle.init(op, rho0), n).sum(0)


def richardson(F, h):
    # central differences at h and h/2 combined to cancel the h^2 term
    D1 = (F(h) - F(-h)) / (2 * h)
    D2 = (F(h / 2) - F(-h / 2)) / h
    return (4 * D2 - D1) / 3


CASES = [
    # (eos, Tr, force, grad, tau, walls)
    ("cs", 0.75, "sc", "hdm", 1.0, False),
    ("pr", 0.9, "zc", "hdm", 0.8, False),
    ("vdw", 0.85, "sc", "cdm", 1.3, False),
    ("rk", 0.85, "zc", "cdm", 1.0, False),
    ("rks", 0.85, "sc", "hdm", 1.0, False),
    ("cs", 0.8, "sc", "hdm", 1.0, True),
]
NSTEPS = 20


@pytest.mark.parametrize("eos,Tr,force,grad,tau,walls", CASES)
def test_real_part_is_the_real_run(eos, Tr, force, grad, tau, walls):
    op = params(eos, Tr, force, grad, tau, walls)
    rho0, _ = droplet(op)
    d = inputs.uniform01(5, rho0.size).reshape(rho0.shape) - 0.5
    r, _ = oracle.tangent(op, rho0, NSTEPS, drho0=d, dTr=1.0)
    ref = final_rho(op, rho0, NSTEPS)
    assert np.max(np.abs(r - ref) / np.abs(ref)) < 1e-14


@pytest.mark.parametrize("eos,Tr,force,grad,tau,walls", CASES)
def test_temperature_derivative_against_richardson_differences(eos, Tr, force, grad, tau, walls):
    op = params(eos, Tr, force, grad, tau, walls)
    rho0, _ = droplet(op)
    _, d = oracle.tangent(op, rho0, NSTEPS, dTr=1.0)
    fd = richardson(lambda e: final_rho(params(eos, Tr + e, force, grad, tau, walls), rho0, NSTEPS), 1e-3 * Tr)
    assert np.abs(d).max() > 0
    assert np.abs(fd - d).max() < 1e-9 * np.abs(d).max()


@pytest.mark.parametrize("eos,Tr,force,grad,tau,walls", CASES)
def test_field_derivative_against_richardson_differences(eos, Tr, force, grad, tau, walls):
    op = params(eos, Tr, force, grad, tau, walls)
    rho0, span = droplet(op)
    dir0 = inputs.uniform01(7, rho0.size).reshape(rho0.shape) - 0.5
    _, d = oracle.tangent(op, rho0, NSTEPS, drho0=dir0)
    fd = richardson(lambda e: final_rho(op, rho0 + e * dir0, NSTEPS), 1e-3 * span)
    assert np.abs(fd - d).max() < 1e-8 * np.abs(d).max()


@pytest.mark.parametrize("force,grad,tau,G", [("sc", "hdm", 1.0, -1.7), ("zc", "hdm", 0.9, -1.6),
                                             ("sc", "cdm", 1.0, -1.7)])
def test_G_derivative_of_the_effective_mass_model(force, grad, tau, G):
    nx, ny = 40, 32
    op = oracle.params_psi(nx, ny, G, tau=tau, force=force, grad=grad)
    rho0, _ = droplet(op, R=9.0)
    _, d = oracle.tangent(op, rho0, NSTEPS, dG=1.0)
    fd = richardson(lambda e: final_rho(oracle.params_psi(nx, ny, G + e, tau=tau, force=force, grad=grad), rho0,
                                        NSTEPS), 1e-3)
    assert np.abs(d).max() > 0
    assert np.abs(fd - d).max() < 1e-9 * np.abs(d).max()
    # G enters the model only through the effective-mass force: the same
    # direction on a Hu-scaled EOS changes nothing (Eq. 22 has no G)
    op2 = params("cs", 0.75)
    _, d2 = oracle.tangent(op2, droplet(op2)[0], 5, dG=1.0)
    assert not d2.any()


def test_sign_mixing_regime_converges_as_h_squared():
    # VdW at k = 1 and Tr = 0.9: U = p - rho/3 is positive in some cells, so
    # Eq. 22 takes both signs and sqrt|U| has its kink inside the run;
    # differences must step smaller than the distance to the kink.
    n, Tr = 10, 0.9
    op = params("vdw", Tr, k=1.0)
    rho0, _ = droplet(op)
    r, d = oracle.tangent(op, rho0, n, dTr=1.0)
    U = op.k * oracle.p_eos(op, r)[0] - r / 3
    assert (U > 0).any() and (U < 0).any()
    errs = []
    for h in (1e-4, 1e-5, 1e-6):
        fd = (final_rho(params("vdw", Tr + h, k=1.0), rho0, n) - final_rho(params("vdw", Tr - h, k=1.0), rho0, n)) / (
            2 * h)
        errs.append(np.abs(fd - d).max() / np.abs(d).max())
    assert errs[0] / errs[1] > 50 and errs[1] / errs[2] > 50
    assert errs[2] < 1e-5


@pytest.mark.parametrize("walls", [False, True])
def test_tangent_conserves_mass(walls):
    op = params("pr", 0.9, "zc", "hdm", 0.8, walls)
    rho0, _ = droplet(op)
    dir0 = inputs.uniform01(9, rho0.size).reshape(rho0.shape) - 0.5
    _, d = oracle.tangent(op, rho0, NSTEPS, drho0=dir0)
    assert abs(d.sum() - dir0.sum()) < 1e-13 * np.abs(dir0).sum()
    _, dT = oracle.tangent(op, rho0, NSTEPS, dTr=1.0)
    assert abs(dT.sum()) < 1e-13 * np.abs(dT).sum()


def test_tangent_is_linear_in_the_direction():
    op = params("rks", 0.85)
    rho0, _ = droplet(op)
    d1 = inputs.uniform01(3, rho0.size).reshape(rho0.shape) - 0.5
    d2 = inputs.uniform01(4, rho0.size).reshape(rho0.shape) - 0.5
    _, a = oracle.tangent(op, rho0, NSTEPS, drho0=d1)
    _, b = oracle.tangent(op, rho0, NSTEPS, drho0=d2)
    _, c = oracle.tangent(op, rho0, NSTEPS, dTr=1.0)
    _, s = oracle.tangent(op, rho0, NSTEPS, drho0=d1 + 2 * d2, dTr=-0.5)
    assert np.abs(s - (a + 2 * b - 0.5 * c)).max() < 1e-12 * np.abs(s).max()
    # the step size does not matter below the square root of the underflow
    _, a2 = oracle.tangent(op, rho0, NSTEPS, drho0=d1, h=1e-60)
    assert np.abs(a2 - a).max() < 1e-13 * np.abs(a).max()


def test_uniform_state_has_no_temperature_derivative():
    op = params("cs", 0.75)
    rho0 = np.full((op.ny, op.nx), 0.2)
    _, d = oracle.tangent(op, rho0, NSTEPS, dTr=1.0)
    assert not d.any()
    _, d1 = oracle.tangent(op, rho0, NSTEPS, drho0=np.ones_like(rho0))
    assert np.abs(d1 - 1.0).max() < 1e-14
