"""GPU tests of the original Shan-Chen effective mass (Eq. 4-5,
psi = 1 - exp(-rho/rho0), eos "psi_exp"): the library runs it through the
Eq. 22 form of U = (G/2) psi^2, the oracle through Eq. 4 literally.  FP64 step
parity (both forces, both gradients), the FP32 single-pass kernel, a batch
instance, and the reverse mode, where the interaction strength G now has a
live gradient (checked against central differences of the FP64 path and of
the oracle)."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()


def pair(nx, ny, G=-1.6, rho0=1.0, force="sc", grad="hdm", tau=1.0, prec="f64"):
    gp = lbm.Params(nx=nx, ny=ny, eos="psi_exp", G=G, rho0=rho0, tau=tau, force=force, grad=grad, prec=prec)
    op = oracle.params_psi(nx, ny, G, rho0=rho0, tau=tau, force=force, grad=grad)
    return gp, op


def droplet_state(op, nx, ny, seed):
    g, l, _ = oracle.maxwell(op)
    rho = inputs.droplet(nx, ny, min(nx, ny) / 4, g, l)
    xi = inputs.uniform01(seed, 2 * nx * ny).reshape(2, ny, nx)
    return oracle.init(op, rho, 0.01 * (xi[0] - 0.5), 0.01 * (xi[1] - 0.5))


GC = lambda rho0: -4.0 * rho0 / 3.0   # critical strength of Eq. 5


@pytest.mark.parametrize("force,grad,tau,G,rho0", [("sc", "hdm", 1.0, -1.6, 1.0), ("zc", "hdm", 0.9, -1.6, 1.0),
                                                   ("sc", "cdm", 1.2, 1.2 * GC(0.8), 0.8),
                                                   ("zc", "cdm", 1.0, 1.2 * GC(1.3), 1.3)])
def test_f64_one_step_parity(force, grad, tau, G, rho0):
    nx, ny = 48, 40
    gp, op = pair(nx, ny, G, rho0, force, grad, tau)
    f0 = droplet_state(op, nx, ny, seed=5)
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        lat.step(1)
        f1 = lat.get_f()
        lat.step(9)
        f10 = lat.get_f()
    o1 = oracle.step(op, f0)
    assert np.max(np.abs(f1 - o1) / np.abs(o1)) < 1e-12
    o10 = oracle.run(op, f0, 10)
    assert np.max(np.abs(f10 - o10) / np.abs(o10)) < 1e-11


@pytest.mark.parametrize("force", ["sc", "zc"])
def test_f32_single_pass_kernel_parity(force):
    nx, ny = 132, 70
    gp, op = pair(nx, ny, -1.6, 1.0, force, "hdm", prec="f32")
    f0 = droplet_state(op, nx, ny, seed=7)
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        lat.set_timing(True)
        lat.step(1)
        assert "fused_step" in lat.timing()["kernels"]
        f1 = lat.get_f()
    o1 = oracle.step(op, f0)
    assert np.max(np.abs(f1 - o1) / o1) < 1e-5


def test_batch_instance_parity():
    gps, ops = zip(*[pair(64, 24, -1.6), pair(40, 36, 1.2 * GC(0.8), 0.8, "zc", "cdm", 0.9)])
    f0 = [droplet_state(op, op.nx, op.ny, seed=k + 3) for k, op in enumerate(ops)]
    with lbm.Batch(list(gps)) as b:
        b.set_f(f0)
        b.step(1)
        f1 = b.get_f()
    for op, a, got in zip(ops, f0, f1):
        ref = oracle.step(op, a)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12


def adjoint(gp, rho0, target, nsteps, C):
    from paper_1712_06079_gb300.autograd import rollout
    dt = torch.float64 if gp.prec == "f64" else torch.float32
    with lbm.Lattice(gp) as lat:
        r0 = torch.tensor(rho0, dtype=dt, device="cuda", requires_grad=True)
        Tr = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
        G = torch.tensor(gp.G, dtype=torch.float64, requires_grad=True)
        rT = rollout(lat, r0, Tr, G, nsteps, C)
        L = ((rT.double() - torch.tensor(target, device="cuda")) ** 2).sum()
        L.backward()
        return float(L.detach()), r0.grad.double().cpu().numpy(), float(Tr.grad), float(G.grad)


def loss(gp, rho0, target, nsteps):
    with lbm.Lattice(gp) as lat:
        r0 = torch.tensor(rho0, dtype=torch.float64, device="cuda")
        rT = torch.empty_like(r0)
        lat.adjoint_forward(r0.data_ptr(), nsteps, nsteps, rT.data_ptr())
        lat.sync()
        return float(((rT - torch.tensor(target, device="cuda")) ** 2).sum())


@pytest.mark.parametrize("force,grad,tau,G", [("sc", "hdm", 1.0, -1.7), ("zc", "hdm", 0.9, -1.6), ("sc", "cdm", 1.0, -1.7)])
def test_adjoint_dG_against_central_differences(force, grad, tau, G):
    nx, ny, n = 48, 40, 40
    gp, op = pair(nx, ny, G, 1.0, force, grad, tau)
    g, l, _ = oracle.maxwell(op)
    rho0 = inputs.droplet(nx, ny, 10, g, l)
    target = inputs.droplet(nx, ny, 11.5, g, l)
    L, gr, gtr, gG = adjoint(gp, rho0, target, n, 7)
    assert gtr == 0.0 and gG != 0.0
    h = 1e-4 * abs(G)
    fd = (loss(lbm.Params(**{**gp.__dict__, "G": G + h}), rho0, target, n) -
          loss(lbm.Params(**{**gp.__dict__, "G": G - h}), rho0, target, n)) / (2 * h)
    assert gG == pytest.approx(fd, rel=1e-4)
    # and against the oracle's own central difference
    ol = lambda GG: float(((oracle.run(oracle.params_psi(nx, ny, GG, force=force, grad=grad, tau=tau),
                                       oracle.init(op, rho0), n).sum(0) - target) ** 2).sum())
    assert gG == pytest.approx((ol(G + h) - ol(G - h)) / (2 * h), rel=1e-4)
    # the field gradient along a seeded direction
    d = inputs.uniform01(11, nx * ny).reshape(ny, nx) - 0.5
    eps = 1e-6
    fdd = (loss(gp, rho0 + eps * d, target, n) - loss(gp, rho0 - eps * d, target, n)) / (2 * eps)
    assert float((gr * d).sum()) == pytest.approx(fdd, rel=1e-4)


@pytest.mark.parametrize("force,grad,tau,G", [("sc", "hdm", 1.0, -1.7), ("zc", "hdm", 0.9, -1.6), ("sc", "cdm", 1.0, -1.7)])
def test_adjoint_dG_matches_complex_step_oracle(force, grad, tau, G):
    # the oracle's complex-step derivative is exact to rounding: a 1e-11 bar
    nx, ny, n = 48, 40, 40
    gp, op = pair(nx, ny, G, 1.0, force, grad, tau)
    g, l, _ = oracle.maxwell(op)
    rho0 = inputs.droplet(nx, ny, 10, g, l)
    target = inputs.droplet(nx, ny, 11.5, g, l)
    L, gr, _, gG = adjoint(gp, rho0, target, n, 7)
    r, dG = oracle.tangent(op, rho0, n, dG=1.0)
    assert L == pytest.approx(float(((r - target) ** 2).sum()), rel=1e-10)
    assert gG == pytest.approx(float((2 * (r - target) * dG).sum()), rel=1e-11)
    d = inputs.uniform01(11, nx * ny).reshape(ny, nx) - 0.5
    _, dd = oracle.tangent(op, rho0, n, drho0=d)
    assert float((gr * d).sum()) == pytest.approx(float((2 * (r - target) * dd).sum()), rel=1e-11)


def test_adjoint_dG_fp32_close_to_fp64():
    nx, ny, n = 128, 96, 100
    gp64, op = pair(nx, ny, -1.7)
    g, l, _ = oracle.maxwell(op)
    rho0 = inputs.droplet(nx, ny, 24, g, l)
    target = inputs.droplet(nx, ny, 26, g, l)
    C = math.ceil(math.sqrt(n))
    L64, g64, _, G64 = adjoint(gp64, rho0, target, n, C)
    L32, g32, _, G32 = adjoint(lbm.Params(**{**gp64.__dict__, "prec": "f32"}), rho0, target, n, C)
    assert L32 == pytest.approx(L64, rel=1e-4)
    assert G32 == pytest.approx(G64, rel=2e-3)
    assert np.abs(g32 - g64).max() < 1e-3 * np.abs(g64).max()
