"""Pins of the oracle's no-slip walls (Sec. 5.5: walls in y, periodic in x).

Readings (the paper gives neither): half-way bounce-back for the no-slip
condition, and the field mirrored across each wall for the gradient (zero
normal gradient), so Eq. 20 along a column is solved on the mirrored column.

Pins, each by another construction than the oracle's:
- HDM: Eq. 20 on the bounded column written out with the reflected ghosts
  (q even, its derivative odd about each wall) as a dense system and solved
  directly;
- CDM: Eq. 15 on an explicitly reflection-padded array;
- no-slip: a shear wave u_x = A sin(pi (y + 1/2) / ny), zero on both walls,
  decays at the Stokes rate nu (pi / ny)^2 with nu = (tau - 1/2) / 3;
- bounce-back conserves mass exactly, and a fluid at rest stays at rest."""
import numpy as np
import pytest

import oracle


def dense_hdm_walls(q):
    # rows i = 0..n-1 of Eq. 20 (h = 1), with q(-1-j) = q(j), q(n+j) = q(n-1-j)
    # and d(-1-j) = -d(j), d(n+j) = -d(n-1-j)
    n = q.size
    A = np.zeros((n, n))
    rhs = np.zeros(n)
    def qq(i):
        if i < 0:
            i = -1 - i
        if i >= n:
            i = 2 * n - 1 - i
        return q[i]
    def add(i, j, c):   # coefficient c on d(j), j possibly a ghost
        if j < 0:
            A[i, -1 - j] -= c
        elif j >= n:
            A[i, 2 * n - 1 - j] -= c
        else:
            A[i, j] += c
    for i in range(n):
        add(i, i - 1, 1 / 3)
        add(i, i, 1.0)
        add(i, i + 1, 1 / 3)
        rhs[i] = 14 / 9 * (qq(i + 1) - qq(i - 1)) / 2 + 1 / 9 * (qq(i + 2) - qq(i - 2)) / 4
    return np.linalg.solve(A, rhs)


@pytest.mark.parametrize("ny", [3, 4, 7, 16, 41])
def test_hdm_walls_against_dense_bounded_solve(ny):
    rng = np.random.default_rng(ny)
    q = rng.random((ny, 5))
    p = oracle.Params(5, ny, grad="hdm", walls=True)
    gx, gy = oracle.grad(p, q)
    for x in range(5):
        assert np.abs(gy[:, x] - dense_hdm_walls(q[:, x])).max() < 1e-13
    # along x nothing changes: the periodic solve of every row
    assert np.abs(gx - oracle.hdm_grad(q)[0]).max() < 1e-15


@pytest.mark.parametrize("ny", [2, 5, 16])
def test_cdm_walls_against_reflection_padding(ny):
    rng = np.random.default_rng(100 + ny)
    nx = 6
    q = rng.random((ny, nx))
    pad = np.pad(np.pad(q, ((1, 1), (0, 0)), mode="symmetric"), ((0, 0), (1, 1)), mode="wrap")
    c = lambda dy, dx: pad[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    ex = (c(0, 1) - c(0, -1)) / 3 + ((c(1, 1) + c(-1, 1)) - (c(1, -1) + c(-1, -1))) / 12
    ey = (c(1, 0) - c(-1, 0)) / 3 + ((c(1, 1) + c(1, -1)) - (c(-1, 1) + c(-1, -1))) / 12
    gx, gy = oracle.grad(oracle.Params(nx, ny, grad="cdm", walls=True), q)
    assert np.abs(gx - ex).max() < 1e-15 and np.abs(gy - ey).max() < 1e-15


def uniform_state(p, rho, ux=None):
    r = np.full((p.ny, p.nx), rho)
    return oracle.init(p, r, ux, None)


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_shear_wave_decays_at_stokes_rate(tau):
    ny, nx, A = 32, 4, 1e-4
    p = oracle.params_at(nx, ny, "cs", 1.0, 4.0, 0.8, k=0.04, tau=tau, walls=True)
    y = np.arange(ny)[:, None] + 0.5
    mode = np.sin(np.pi * y / ny) * np.ones((1, nx))
    f = uniform_state(p, 0.3, A * mode)
    amp = []
    for t0, t1 in ((0, 200), (200, 600)):
        f = oracle.run(p, f, t1 - t0)
        rho, vx, vy = oracle.moments(p, f)
        amp.append(float((vx * mode).sum() / (mode * mode).sum()))
    rate = np.log(amp[0] / amp[1]) / 400
    nu = (tau - 0.5) / 3
    assert rate == pytest.approx(nu * (np.pi / ny) ** 2, rel=0.02)


def test_walls_conserve_mass_and_keep_rest():
    nx, ny = 40, 30
    p = oracle.params_at(nx, ny, "cs", 1.0, 4.0, 0.8, k=0.04, tau=0.9, walls=True)
    g, l, _ = oracle.maxwell(p)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    rho = g + (l - g) * 0.5 * (1 - np.tanh((np.hypot(X - 20, Y - 8) - 7) / 2))   # drop touching the wall
    f0 = oracle.init(p, rho)
    m0 = f0.sum()
    f = oracle.run(p, f0, 200)
    assert abs(f.sum() - m0) < 1e-12 * m0
    assert np.isfinite(f).all()
    # a uniform fluid at rest between the walls stays exactly at rest
    f1 = uniform_state(p, 0.25)
    assert np.abs(oracle.run(p, f1, 50) - f1).max() < 1e-15
