"""GPU tests of the reverse-mode (adjoint) step: gradients of
L = sum (rho_T - rho_target)^2 with respect to the initial density field and
the reduced temperature, against central finite differences of the FP64 GPU
path and of the FP64 oracle and against the oracle's complex-step derivative
(exact to rounding, so the bar is 1e-11 instead of the differences' 1e-4), for
both force forms, both gradients and tau != 1; checkpoint intervals must not
change the result; dL/dG = 0."""
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


T = inputs.EOS_TABLE


def setup(nx, ny, eos, Tr, force="sc", grad="hdm", tau=1.0, prec="f64", R0=None, R1=None):
    t = T[eos]
    p = lbm.Params(nx=nx, ny=ny, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=Tr, k=t["k"], tau=tau,
                   force=force, grad=grad, prec=prec, stream=torch.cuda.current_stream().cuda_stream)
    g, l = lbm.maxwell(p)
    R0 = R0 or min(nx, ny) / 4
    R1 = R1 or R0 * 9 / 8
    rho0 = inputs.droplet(nx, ny, R0, g, l)
    target = inputs.droplet(nx, ny, R1, g, l)
    return p, rho0, target


def loss_of(p, rho0, target, nsteps):
    dt = torch.float64 if p.prec == "f64" else torch.float32
    with lbm.Lattice(p) as lat:
        r0 = torch.tensor(rho0, dtype=dt, device="cuda")
        rT = torch.empty_like(r0)
        lat.adjoint_forward(r0.data_ptr(), nsteps, nsteps, rT.data_ptr())
        lat.sync()
        return float(((rT.double() - torch.tensor(target, device="cuda")) ** 2).sum())


def adjoint(p, rho0, target, nsteps, C):
    from paper_1712_06079_gb300.autograd import rollout
    dt = torch.float64 if p.prec == "f64" else torch.float32
    with lbm.Lattice(p) as lat:
        r0 = torch.tensor(rho0, dtype=dt, device="cuda", requires_grad=True)
        Tr = torch.tensor(p.Tr, dtype=torch.float64, requires_grad=True)
        G = torch.tensor(-1.0, dtype=torch.float64, requires_grad=True)
        rT = rollout(lat, r0, Tr, G, nsteps, C)
        L = ((rT.double() - torch.tensor(target, device="cuda")) ** 2).sum()
        L.backward()
        return float(L.detach()), r0.grad.double().cpu().numpy(), float(Tr.grad), float(G.grad)


CASES = [
    ("cs", 0.75, "sc", "hdm", 1.0, 48, 40),
    ("pr", 0.9, "zc", "hdm", 0.8, 40, 36),   # ZC at lower Tr goes unstable within 40 steps (oracle too)
    ("vdw", 0.85, "sc", "cdm", 1.3, 36, 36),
    ("rk", 0.85, "zc", "cdm", 1.0, 40, 32),
]


@pytest.mark.parametrize("eos,Tr,force,grad,tau,nx,ny", CASES)
def test_adjoint_against_central_differences_fp64(eos, Tr, force, grad, tau, nx, ny):
    nsteps = 40
    p, rho0, target = setup(nx, ny, eos, Tr, force, grad, tau)
    L, g_rho0, g_tr, g_G = adjoint(p, rho0, target, nsteps, 7)
    assert g_G == 0.0
    # temperature: central difference, h = 1e-4 (relative to Tr)
    h = 1e-4 * Tr
    pp, pm = lbm.Params(**{**p.__dict__, "Tr": Tr + h}), lbm.Params(**{**p.__dict__, "Tr": Tr - h})
    fd_tr = (loss_of(pp, rho0, target, nsteps) - loss_of(pm, rho0, target, nsteps)) / (2 * h)
    assert g_tr == pytest.approx(fd_tr, rel=1e-4, abs=1e-10 * abs(L))
    # initial field: directional derivative along a seeded direction
    d = inputs.uniform01(7, nx * ny).reshape(ny, nx) - 0.5
    eps = 1e-6 * np.abs(rho0).max()
    fd_dir = (loss_of(p, rho0 + eps * d, target, nsteps) - loss_of(p, rho0 - eps * d, target, nsteps)) / (2 * eps)
    assert float((g_rho0 * d).sum()) == pytest.approx(fd_dir, rel=1e-4)


@pytest.mark.parametrize("eos,Tr,force,grad,tau,nx,ny", CASES)
def test_adjoint_matches_complex_step_oracle(eos, Tr, force, grad, tau, nx, ny):
    nsteps = 40
    p, rho0, target = setup(nx, ny, eos, Tr, force, grad, tau)
    L, g_rho0, g_tr, _ = adjoint(p, rho0, target, nsteps, 7)
    t = T[eos]
    op = oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=t["k"], tau=tau, force=force,
                          grad=grad)
    # dL/dtheta = sum 2 (rho_T - target) d rho_T/dtheta, d rho_T from the complex step
    r, dT = oracle.tangent(op, rho0, nsteps, dTr=1.0)
    assert L == pytest.approx(float(((r - target) ** 2).sum()), rel=1e-10)
    assert g_tr == pytest.approx(float((2 * (r - target) * dT).sum()), rel=1e-11)
    d = inputs.uniform01(7, nx * ny).reshape(ny, nx) - 0.5
    _, dd = oracle.tangent(op, rho0, nsteps, drho0=d)
    assert float((g_rho0 * d).sum()) == pytest.approx(float((2 * (r - target) * dd).sum()), rel=1e-11)
    # and cell by cell at a few cells (unit directions)
    for (y, x) in [(ny // 2, nx // 2), (ny // 2, nx // 2 + 9), (3, 4)]:
        e = np.zeros_like(rho0)
        e[y, x] = 1.0
        _, de = oracle.tangent(op, rho0, nsteps, drho0=e)
        assert g_rho0[y, x] == pytest.approx(float((2 * (r - target) * de).sum()), rel=1e-10,
                                             abs=1e-12 * np.abs(g_rho0).max())


def test_adjoint_matches_oracle_finite_differences():
    # the FP64 oracle's own gradient (central differences of its forward run)
    nx, ny, nsteps, Tr = 32, 28, 30, 0.75
    p, rho0, target = setup(nx, ny, "cs", Tr)
    L, g_rho0, g_tr, _ = adjoint(p, rho0, target, nsteps, 5)
    t = T["cs"]

    def oracle_loss(tr, r0):
        op = oracle.params_at(nx, ny, "cs", t["a"], t["b"], tr, k=t["k"])
        f = oracle.run(op, oracle.init(op, r0), nsteps)
        return float(((f.sum(0) - target) ** 2).sum())

    h = 1e-4 * Tr
    fd = (oracle_loss(Tr + h, rho0) - oracle_loss(Tr - h, rho0)) / (2 * h)
    assert g_tr == pytest.approx(fd, rel=1e-4)
    assert L == pytest.approx(oracle_loss(Tr, rho0), rel=1e-10)
    # field gradient at a few cells by central differences of the oracle
    for (y, x) in [(ny // 2, nx // 2), (ny // 2, nx // 2 + 9), (3, 4)]:
        e = np.zeros_like(rho0)
        e[y, x] = 1.0
        eps = 1e-6
        fd = (oracle_loss(Tr, rho0 + eps * e) - oracle_loss(Tr, rho0 - eps * e)) / (2 * eps)
        assert g_rho0[y, x] == pytest.approx(fd, rel=1e-4, abs=1e-9 * np.abs(g_rho0).max())


def test_checkpoint_interval_does_not_change_the_gradient():
    p, rho0, target = setup(40, 40, "cs", 0.8)
    ref = adjoint(p, rho0, target, 25, 1)
    for C in (4, 5, 25):
        L, g, gtr, _ = adjoint(p, rho0, target, 25, C)
        assert L == ref[0]
        assert np.array_equal(g, ref[1]) and gtr == ref[2]


def test_single_pass_records_give_the_same_gradient_for_every_checkpoint_interval():
    # FP32 single-pass layout: the reverse sweep reads the forward kernel's
    # records (the last two segments' from the taped forward, the others
    # recomputed), so the gradient must not depend on the interval, down to the
    # bit, including C = 1, an interval that does not divide N and C > N
    p, rho0, target = setup(64, 64, "cs", 0.75, prec="f32", R0=16, R1=18)
    ref = adjoint(p, rho0, target, 25, 25)
    for C in (1, 2, 4, 7, 13, 40):
        L, g, gtr, _ = adjoint(p, rho0, target, 25, C)
        assert L == ref[0]
        assert np.array_equal(g, ref[1]) and gtr == ref[2], C


def test_second_backward_after_one_forward_recomputes_the_same_gradient():
    # the first sweep starts from the taped segments, the second recomputes them
    for prec, C in (("f32", 6), ("f64", 6), ("f32", 50)):
        p, rho0, target = setup(64, 64, "cs", 0.75, prec=prec, R0=16, R1=18)
        dt = torch.float64 if prec == "f64" else torch.float32
        with lbm.Lattice(p) as lat:
            r0 = torch.tensor(rho0, dtype=dt, device="cuda")
            rT = torch.empty_like(r0)
            lat.adjoint_forward(r0.data_ptr(), 40, C, rT.data_ptr())
            lat.sync()
            gr = (2 * (rT.double() - torch.tensor(target, device="cuda"))).to(dt).contiguous()
            outs = []
            for _ in range(2):
                g0 = torch.empty_like(r0)
                _, gtr, _ = lat.adjoint_backward(gr.data_ptr(), g0.data_ptr())
                outs.append((g0.cpu().numpy(), gtr))
        assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1], (prec, C)


def test_adjoint_fp32_close_to_fp64():
    p64, rho0, target = setup(64, 64, "cs", 0.75, R0=16, R1=18)
    p32 = lbm.Params(**{**p64.__dict__, "prec": "f32"})
    n = 100
    C = math.ceil(math.sqrt(n))
    L64, g64, t64, _ = adjoint(p64, rho0, target, n, C)
    L32, g32, t32, _ = adjoint(p32, rho0, target, n, C)
    assert L32 == pytest.approx(L64, rel=1e-4)
    assert t32 == pytest.approx(t64, rel=1e-3)
    assert np.abs(g32 - g64).max() < 1e-3 * np.abs(g64).max()


FP32_CASES = [
    # (eos, Tr, force, grad, tau, nx, ny): the single-pass layout with tau != 1
    # (nine-field lambda), ragged 64 x 16 adjoint tiles, and the plain-layout
    # FP32 path (CDM)
    ("cs", 0.8, "sc", "hdm", 0.8, 100, 70),
    ("pr", 0.9, "zc", "hdm", 1.0, 132, 58),
    ("vdw", 0.85, "sc", "cdm", 1.2, 48, 40),
]


@pytest.mark.parametrize("eos,Tr,force,grad,tau,nx,ny", FP32_CASES)
def test_adjoint_fp32_paths_close_to_fp64(eos, Tr, force, grad, tau, nx, ny):
    p64, rho0, target = setup(nx, ny, eos, Tr, force, grad, tau)
    p32 = lbm.Params(**{**p64.__dict__, "prec": "f32"})
    n = 30
    L64, g64, t64, _ = adjoint(p64, rho0, target, n, 6)
    L32, g32, t32, _ = adjoint(p32, rho0, target, n, 6)
    assert L32 == pytest.approx(L64, rel=1e-4)
    assert t32 == pytest.approx(t64, rel=2e-3)
    assert np.abs(g32 - g64).max() < 1e-3 * np.abs(g64).max()
