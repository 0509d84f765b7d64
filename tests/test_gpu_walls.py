"""GPU: no-slip walls in y (Sec. 5.5) through the C ABI against the FP64
oracle's walled step (half-way bounce-back, field mirrored across the walls).

Bars as in the periodic parity tests: FP64 within 1e-12 relative per step over
all nine populations and over 20 steps; FP32 within 1e-5 on rho after 300
steps; mass conserved to FP64 rounding.  Walled FP32 lattices that the
single-pass kernel takes run it, the others the two-pass kernels; the batch
and the reverse mode refuse walls."""
import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu
EOS = dict(inputs.EOS_TABLE)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()


def make(nx, ny, eos="cs", Tr=0.8, force="sc", grad="hdm", tau=1.0, prec="f64"):
    t = EOS[eos]
    gp = lbm.Params(nx=nx, ny=ny, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=Tr, k=t["k"], tau=tau,
                    force=force, grad=grad, prec=prec, walls=True)
    op = oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=t["k"], tau=tau, force=force,
                          grad=grad, walls=True)
    return gp, op


def wall_drop(op, nx, ny, seed):
    # a droplet resting on the bottom wall, a film along the top wall, small seeded velocities
    g, l, _ = oracle.maxwell(op)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    r = min(nx, ny) / 4
    drop = 0.5 * (1 - np.tanh((np.hypot(X - nx / 2, Y - r * 0.6) - r) / 2))
    film = 0.5 * (1 + np.tanh((Y - (ny - 1 - max(2, ny // 8))) / 2))
    rho = g + (l - g) * np.clip(drop + film, 0, 1)
    xi = inputs.uniform01(seed, 2 * nx * ny).reshape(2, ny, nx)
    return oracle.init(op, rho, 0.01 * (xi[0] - 0.5), 0.01 * (xi[1] - 0.5))


CASES = [
    # (nx, ny, eos, Tr, force, grad, tau)
    (96, 64, "cs", 0.8, "sc", "hdm", 1.0),
    (64, 40, "pr", 0.75, "zc", "hdm", 0.8),
    (70, 36, "vdw", 0.85, "sc", "cdm", 1.2),
    (40, 8, "cs", 0.8, "zc", "hdm", 1.0),     # mirrored column shorter than the stencil: folded
    (33, 21, "rk", 0.8, "sc", "hdm", 0.9),    # ragged tiles
]


@pytest.mark.parametrize("nx,ny,eos,Tr,force,grad,tau", CASES)
def test_f64_walls_parity(nx, ny, eos, Tr, force, grad, tau):
    gp, op = make(nx, ny, eos, Tr, force, grad, tau)
    f0 = wall_drop(op, nx, ny, seed=nx + 7 * ny)
    with lbm.Lattice(gp) as lat:
        assert lat.segment_rows() == 0          # the two-pass kernels
        lat.set_f(f0)
        lat.step(1)
        f1 = lat.get_f()
        lat.step(19)
        f20 = lat.get_f()
    o1 = oracle.step(op, f0)
    assert (np.abs(f1 - o1) / np.abs(o1)).max() < 1e-12
    o20 = oracle.run(op, o1, 19)
    assert (np.abs(f20 - o20) / np.abs(o20)).max() < 1e-11
    assert abs(f20.sum() - f0.sum()) < 1e-13 * f0.sum()


@pytest.mark.parametrize("two_pass", [False, True])
def test_f32_walls_parity(two_pass):
    # 128 x 72 runs the single-pass kernel (walls in its staging and its
    # push), or the two-pass kernels with LBM_FLAG_TWO_PASS
    nx, ny = 128, 72
    gp, op = make(nx, ny, "cs", 0.8, "sc", "hdm", 0.9, prec="f32")
    gp.two_pass = two_pass
    f0 = wall_drop(op, nx, ny, seed=3)
    with lbm.Lattice(gp) as lat:
        assert (lat.segment_rows() > 0) == (not two_pass)
        lat.set_f(f0)
        lat.set_timing(True)
        lat.step(1)
        assert ("fused_step" in lat.timing()["kernels"]) == (not two_pass)
        f1 = lat.get_f()
        lat.step(299)
        r, _, _ = lat.moments()
        obs = lat.observables()
    o1 = oracle.step(op, f0)
    assert np.max(np.abs(f1 - o1) / o1) < 1e-5
    ro, _, _ = oracle.moments(op, oracle.run(op, o1, 299))
    assert np.max(np.abs(r - ro) / ro) < 1e-5
    assert abs(obs["mass"] - ro.sum()) < 1e-6 * ro.sum()


@pytest.mark.parametrize("nx,ny,eos,force,tau,grad", [(132, 129, "pr", "zc", 1.0, "hdm"), (64, 54, "vdw", "sc", 0.8, "hdm"),
                                                      (256, 200, "cs", "sc", 1.0, "hdm"), (132, 70, "vdw", "sc", 1.0, "cdm"),
                                                      (64, 54, "vdw", "zc", 0.8, "cdm")])
def test_f32_walls_single_pass_one_step_and_segments(nx, ny, eos, force, tau, grad):
    # one step of the single-pass kernel with walls against the oracle, every
    # population, at several segment heights (segments start and end at the
    # walls and inside the lattice); HDM and the CDM variant
    gp, op = make(nx, ny, eos, 0.8, force, grad, tau, prec="f32")
    f0 = wall_drop(op, nx, ny, seed=nx + ny)
    fo = oracle.step(op, f0)
    for rows in (0, 6, 22, ny):
        with lbm.Lattice(gp) as lat:
            lat.set_segment_rows(rows)
            assert lat.segment_rows() > 0
            lat.set_f(f0)
            lat.step(1)
            f1 = lat.get_f()
        assert np.max(np.abs(f1 - fo) / fo) < 1e-5, rows


@pytest.mark.parametrize("grad", ["hdm", "cdm"])
@pytest.mark.parametrize("ny", [5, 48])
def test_gradient_with_walls(grad, ny):
    nx = 24
    gp, op = make(nx, ny, grad=grad)
    xi = inputs.uniform01(ny + 11, nx * ny).reshape(ny, nx)
    with lbm.Lattice(gp) as lat:
        gx, gy = lat.gradient(xi, 0.5)
    ox, oy = oracle.grad(op, xi)
    scale = max(np.abs(ox).max(), np.abs(oy).max())
    assert np.abs(gx - ox / 0.5).max() < 1e-12 * scale
    assert np.abs(gy - oy / 0.5).max() < 1e-12 * scale


def test_walls_refused_where_unsupported():
    torch = pytest.importorskip("torch")
    gp, _ = make(64, 32)
    with lbm.Lattice(gp) as lat:
        x = torch.full((32, 64), 0.3, dtype=torch.float64, device="cuda")
        r = torch.empty_like(x)
        with pytest.raises(lbm.LBMError) as ei:
            lat.adjoint_forward(x.data_ptr(), 10, 3, r.data_ptr())
        assert ei.value.status == lbm.E_INVALID
    with pytest.raises(lbm.LBMError):
        lbm.Batch([gp, gp])


def test_splash_small_spreads_and_forces_agree():
    # the Sec. 5.5 set-up at a fifth of the size (200 x 60, film 6, R 10,
    # U 0.1), PR at T/Tc = 0.7, tau = 1 (Re = U D / nu = 12): stable, mass conserved, the
    # liquid spreads along the film after impact, and the Shan-Chen (Eq. 22)
    # and Zhang-Chen (Eq. 7) forms, the same force, give the same spread
    t = EOS["pr"]
    nx, ny, film, R, U = 200, 60, 6, 10, 0.1
    g, l = lbm.maxwell(lbm.Params(nx=8, ny=8, eos="pr", a=t["a"], b=t["b"], omega=t["omega"], Tr=0.7, k=t["k"]))
    rho, ux, uy = inputs.splash(nx, ny, film, R, U, g, l, 4.0)
    tau = 1.0
    widths = {}
    for force in ("sc", "zc"):
        p = lbm.Params(nx=nx, ny=ny, eos="pr", a=t["a"], b=t["b"], omega=t["omega"], Tr=0.7, k=t["k"], tau=tau,
                       force=force, grad="hdm", prec="f32", walls=True)
        with lbm.Lattice(p) as lat:
            lat.init_density(rho, ux, uy)
            w = []
            for _ in range(8):
                lat.step(40)
                r, _, _ = lat.moments()
                w.append(int(np.count_nonzero(r[film + 1] > 0.5 * (g + l))))
            obs = lat.observables()
        assert abs(obs["mass"] - rho.sum()) < 1e-5 * rho.sum()
        widths[force] = w
    assert widths["sc"][0] == 0 or widths["sc"][0] < widths["sc"][-1]
    assert widths["sc"][-1] > widths["sc"][2] > 0        # spreads along the film after contact
    assert max(abs(a - b) for a, b in zip(widths["sc"], widths["zc"])) <= 2
