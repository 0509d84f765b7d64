"""Pins of the oracle's derivative operators: the HDM compact scheme of Eq. 20
(periodic, solved by cyclic Thomas) and the weighted CDM of Eq. 15.

Pins: the Fourier symbol of Eq. 20 (closed form), a dense LU solve on tiny
lattices (brute force), sixth-order convergence, and the tanh study of
Sec. 3 (Figs. 1-3: HDM error below CDM error for every interface width)."""
import numpy as np
import pytest

import oracle


def hdm_symbol(theta):
    # Substituting u = exp(i theta x) into Eq. 20 (h = 1):
    #   d (1 + (2/3) cos th) = i [(14/9) sin th + (1/18) sin 2th] u
    return (14 / 9 * np.sin(theta) + 1 / 18 * np.sin(2 * theta)) / (1 + 2 / 3 * np.cos(theta))


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8, 9, 16, 33, 64, 257])
def test_hdm_fourier_modes(n):
    x = np.arange(n)
    for m in range(0, n // 2 + 1):
        th = 2 * np.pi * m / n
        for phase in (0.0, 0.7):
            u = np.sin(th * x + phase)
            d = oracle.hdm_line(u)
            exact = hdm_symbol(th) * np.cos(th * x + phase)
            assert np.allclose(d, exact, rtol=0, atol=1e-12), (n, m)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 11, 16])
def test_hdm_dense_bruteforce(n):
    # dense periodic system of Eq. 20 solved by LU (numpy), random data
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n)
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for i in range(n):
        A[i, i] += 1.0
        A[i, (i - 1) % n] += 1 / 3
        A[i, (i + 1) % n] += 1 / 3
        B[i, (i + 2) % n] += 1 / 36
        B[i, (i - 2) % n] -= 1 / 36
        B[i, (i + 1) % n] += 7 / 9
        B[i, (i - 1) % n] -= 7 / 9
    ref = np.linalg.solve(A, B @ u)
    assert np.allclose(oracle.hdm_line(u), ref, rtol=0, atol=1e-13)


def test_hdm_sixth_order_convergence():
    # error of d/dx sin(2 pi x / N) falls as N^-6
    errs = []
    for n in (16, 32, 64):
        x = np.arange(n)
        k = 2 * np.pi / n
        d = oracle.hdm_line(np.sin(k * x))
        errs.append(np.max(np.abs(d - k * np.cos(k * x))) / k)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 55 < r1 < 70 and 60 < r2 < 68


def test_hdm_antisymmetric_and_constant():
    rng = np.random.default_rng(1)
    n = 37
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    # the periodic operator is an antisymmetric circulant: <v, D u> = -<D v, u>
    assert np.dot(v, oracle.hdm_line(u)) == pytest.approx(-np.dot(oracle.hdm_line(v), u), abs=1e-12)
    assert np.all(oracle.hdm_line(np.full(n, 3.7)) == 0.0)


def test_hdm_2d_separable():
    ny, nx = 12, 20
    y, x = np.mgrid[0:ny, 0:nx]
    tx, ty = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    q = np.sin(tx * x) * np.cos(ty * y)
    gx, gy = oracle.hdm_grad(q)
    assert np.allclose(gx, hdm_symbol(tx) * np.cos(tx * x) * np.cos(ty * y), atol=1e-13)
    assert np.allclose(gy, -hdm_symbol(ty) * np.sin(tx * x) * np.sin(ty * y), atol=1e-13)


def test_cdm_plane_wave():
    # Eq. 15 times 1/c_s^2 on q = sin(th x + ph y):
    #   d/dx = [(2/3) + (1/3) cos ph] sin th cos(th x + ph y) (and x <-> y);
    # for ph = 0 it is the 1-D central difference of Eq. 14.
    ny, nx = 10, 14
    y, x = np.mgrid[0:ny, 0:nx]
    for mx, my in [(1, 0), (2, 3), (5, 4), (7, 5)]:
        th, ph = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
        q = np.sin(th * x + ph * y)
        gx, gy = oracle.cdm_grad(q)
        c = np.cos(th * x + ph * y)
        assert np.allclose(gx, (2 / 3 + np.cos(ph) / 3) * np.sin(th) * c, atol=1e-13)
        assert np.allclose(gy, (2 / 3 + np.cos(th) / 3) * np.sin(ph) * c, atol=1e-13)


def tanh_errors(width, n=512, window=10):
    # Eq. 16 on a periodic slab: rho = 1 + tanh(2(x - x1)/W) - tanh(2(x - x2)/W)
    x = np.arange(n, dtype=float)
    x1, x2 = n / 4, 3 * n / 4
    rho = 1 + np.tanh(2 * (x - x1) / width) - np.tanh(2 * (x - x2) / width)
    exact = (2 / width) * (np.tanh(2 * (x - x2) / width) ** 2 - np.tanh(2 * (x - x1) / width) ** 2)  # sech^2 = 1 - tanh^2
    sel = np.abs(x - x1) <= window
    d_h = oracle.hdm_line(rho)
    d_c = oracle.cdm_grad(np.tile(rho, (3, 1)))[0][1]
    err = lambda d: np.sqrt(np.mean((d[sel] - exact[sel]) ** 2))  # Eq. 18
    return err(d_c), err(d_h)


@pytest.mark.parametrize("width", [1.0, 2.0, 3.0, 4.0, 5.0])
def test_tanh_hdm_beats_cdm(width):
    # Sec. 3: for every interface width, the HDM standard error (Eq. 18) is
    # below the CDM one, and the gap widens with W (Fig. 3)
    e_c, e_h = tanh_errors(width)
    assert e_h < e_c
    if width >= 3:
        assert e_h < 0.2 * e_c
