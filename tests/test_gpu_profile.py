"""GPU: the gradient operator through the C ABI (lbm_gradient) against the
FP64 oracle, and the flat-interface study of Sec. 5.1 (Fig. 4): on the exact
equilibrium profile of the VdW fluid at T/Tc = 0.9 (h = 0.5) the HDM derivative
of the CUDA path is far closer to the exact slope than the CDM one.

Bars: FP64 within 1e-12 of the oracle's cyclic solve of Eq. 20 (and of Eq. 15
for CDM) relative to the largest derivative; FP32 within 2e-6 of the field's
magnitude (the field and the sum rounded to FP32)."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()


def lattice(nx, ny, grad="hdm", prec="f64"):
    return lbm.Lattice(lbm.Params(nx=nx, ny=ny, eos="cs", a=1.0, b=4.0, Tr=0.8, force="sc", grad=grad, prec=prec))


@pytest.mark.parametrize("nx,ny", [(64, 48), (100, 8), (9, 130), (3, 5)])
@pytest.mark.parametrize("grad", ["hdm", "cdm"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("h", [1.0, 0.5])
def test_gradient_matches_oracle(nx, ny, grad, prec, h):
    # seeded smooth-plus-rough periodic field: every tap of the stencil matters
    xi = inputs.uniform01(7 + nx + 3 * ny, nx * ny).reshape(ny, nx)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    q = 1.0 + 0.3 * np.sin(2 * np.pi * X / nx) * np.cos(4 * np.pi * Y / ny) + 0.05 * (xi - 0.5)
    ox, oy = (oracle.hdm_grad if grad == "hdm" else oracle.cdm_grad)(q)
    ox, oy = ox / h, oy / h
    with lattice(nx, ny, grad, prec) as lat:
        gx, gy = lat.gradient(q, h)
    if prec == "f64":
        scale = max(np.abs(ox).max(), np.abs(oy).max())
        assert np.abs(gx - ox).max() <= 1e-12 * scale
        assert np.abs(gy - oy).max() <= 1e-12 * scale
    else:
        bar = 2e-6 * np.abs(q).max() / h
        assert np.abs(gx - ox).max() <= bar
        assert np.abs(gy - oy).max() <= bar


def test_gradient_rejects_bad_arguments():
    with lattice(16, 16) as lat:
        with pytest.raises(lbm.LBMError) as ei:
            lat.gradient(np.ones((16, 16)), 0.0)
        assert ei.value.status == lbm.E_INVALID
        with pytest.raises(ValueError):
            lat.gradient(np.ones((8, 16)), 1.0)


def golden_line():
    rows = np.loadtxt(os.path.join(HERE, "golden", "flat_profile_vdw_tr09.txt"))
    rho, drho = rows[:, 1], rows[:, 2]
    # periodic by the mirror image: two interfaces 256 length units apart
    return np.concatenate([rho, rho[::-1]]), np.concatenate([drho, -drho[::-1]])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fig4_flat_interface_hdm_vs_cdm(prec):
    line, exact = golden_line()
    h, n = 0.5, line.size
    q = np.tile(line[:, None], (1, 4))            # the profile along y, uniform in x
    err = {}
    for grad in ("hdm", "cdm"):
        with lattice(4, n, grad, prec) as lat:
            gx, gy = lat.gradient(q, h)
        assert np.abs(gx).max() <= (1e-12 if prec == "f64" else 1e-5)
        d = gy[:, 0]
        err[grad] = np.abs(d - exact).max() / np.abs(exact).max()
        if prec == "f64":   # the same numbers as the oracle's operators on the same line
            ref = oracle.hdm_line(line) / h if grad == "hdm" else oracle.cdm_grad(q)[1][:, 0] / h
            assert np.abs(d - ref).max() <= 1e-12 * np.abs(exact).max()
    assert err["hdm"] < 2e-4
    assert err["cdm"] > 1e-2
    assert err["cdm"] > 100 * err["hdm"]
