"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point ``include/*.h`` declares, validates
parameters before touching the device, and its host-only set-up math agrees
with the oracle (critical points; the explicit HDM weights reproduce the
oracle's cyclic tridiagonal solve of Eq. 20)."""
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "lbm_create" in names and "lbm_step" in names and "lbm_destroy" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding knows the signature of each
    assert set(names) <= set(lbm.SIGNATURES), set(names) - set(lbm.SIGNATURES)


@pytest.mark.parametrize("eos,a,b", [("vdw", 9 / 49, 2 / 21), ("cs", 1.0, 4.0), ("pr", 2 / 49, 2 / 21),
                                     ("rk", 2 / 49, 2 / 21), ("rks", 9 / 49, 2 / 21), ("cs", 0.3, 1.7)])
def test_critical_point_matches_oracle(lib, eos, a, b):
    Tc, rc = lbm.critical_point(eos, a, b)
    To, ro = oracle.critical_point(eos, a, b)
    assert Tc == pytest.approx(To, rel=1e-13)
    assert rc == pytest.approx(ro, rel=1e-7)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 40, 81, 128, 1000])
def test_hdm_weights_reproduce_cyclic_solve(lib, n):
    # the explicit folded stencil equals the exact periodic solve of Eq. 20
    for radius in (40, 48):
        w, ke = lbm.hdm_weights(n, radius)
        assert ke == min(radius, (n - 1) // 2)
        rng = np.random.default_rng(n)
        u = rng.standard_normal(n)
        d = np.zeros(n)
        for j in range(1, ke + 1):
            d += w[j] * (np.roll(u, -j) - np.roll(u, j))
        assert np.allclose(d, oracle.hdm_line(u), rtol=0, atol=5e-15 * max(1, np.abs(u).max()) * 10)


def test_hdm_weights_known_values(lib):
    # N = 8 folds to rational weights [221, -75, 25]/252 (and 0 at j = 4)
    w, ke = lbm.hdm_weights(8, 40)
    assert ke == 3
    assert np.allclose(w[1:4], np.array([221, -75, 25]) / 252, rtol=0, atol=1e-15)
    # long lines: consistency sum_j 2 j w_j = 1 (exact first derivative of a line)
    w, ke = lbm.hdm_weights(4096, 40)
    assert np.sum(2 * np.arange(41) * w) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-1), dict(tau=0.5), dict(Tr=0.0), dict(hdm_radius=49),
                                 dict(b=0.0), dict(prec="bogus")])
def test_create_rejects_bad_params_before_device_work(lib, bad):
    p = lbm.Params(nx=16, ny=16)
    if bad.get("prec") == "bogus":
        c = p.c()
        c.prec = 7
    else:
        for k, v in bad.items():
            setattr(p, k, v)
        c = p.c()
    import ctypes
    h = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(c), ctypes.byref(h))
    assert st == lbm.E_INVALID
    assert h.value is None
    assert lib.lbm_last_error(None)


def test_batch_create_rejects_oversize_totals_before_device_work(lib):
    # device offsets are int cell indices: instances of 2^30 cells each (the
    # per-instance maximum) pass alone, but two of them pad to 2^31 cells and
    # the batch is refused before any allocation
    import ctypes
    one = lbm.Params(nx=32768, ny=32768, eos="cs", Tr=0.8, k=0.04)
    arr = (lbm._Params * 2)(one.c(), one.c())
    h = ctypes.c_void_p()
    assert lib.lbm_batch_create(arr, 2, ctypes.byref(h)) == lbm.E_INVALID
    assert h.value is None
    big = lbm.Params(nx=32769, ny=32768, eos="cs", Tr=0.8, k=0.04)   # one instance over 2^30
    arr1 = (lbm._Params * 1)(big.c())
    assert lib.lbm_batch_create(arr1, 1, ctypes.byref(h)) == lbm.E_INVALID
    assert lib.lbm_batch_create(arr1, 0, ctypes.byref(h)) == lbm.E_INVALID


def test_null_handles_are_safe(lib):
    import ctypes
    lib.lbm_destroy(None)
    assert lib.lbm_step(None, 1) == lbm.E_INVALID
    assert lib.lbm_sync(None) == lbm.E_INVALID
    assert lib.lbm_create(None, None) == lbm.E_INVALID
    assert lib.lbm_last_error(None)


@pytest.mark.parametrize("eos,Tr", [("vdw", 0.5), ("vdw", 0.95), ("cs", 0.7), ("cs", 0.8), ("pr", 0.55), ("pr", 0.9),
                                    ("rk", 0.6), ("rks", 0.75)])
def test_library_maxwell_matches_oracle(lib, eos, Tr):
    from paper_1712_06079_gb300 import inputs
    t = dict(inputs.EOS_TABLE.get(eos, dict(a=9 / 49, b=2 / 21, omega=0.344, k=0.01)))
    g, l = lbm.maxwell(lbm.Params(nx=1, ny=1, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=Tr))
    op = oracle.params_at(1, 1, eos, t["a"], t["b"], Tr, omega=t["omega"])
    go, lo, _ = oracle.maxwell(op)
    assert g == pytest.approx(go, rel=1e-9)
    assert l == pytest.approx(lo, rel=1e-10)


def test_library_maxwell_rejects_supercritical(lib):
    with pytest.raises(lbm.LBMError):
        lbm.maxwell(lbm.Params(nx=1, ny=1, eos="vdw", a=9 / 49, b=2 / 21, Tr=1.02))


@pytest.mark.parametrize("G,rho0", [(-1.6, 1.0), (-2.0, 1.0), (-3.0, 0.5)])
def test_library_maxwell_psi_exp_matches_oracle(lib, G, rho0):
    # the equal-area pair of the pressure of Eq. 5 (original effective mass)
    g, l = lbm.maxwell(lbm.Params(nx=1, ny=1, eos="psi_exp", G=G, rho0=rho0))
    go, lo, _ = oracle.maxwell(oracle.params_psi(1, 1, G, rho0=rho0))
    assert g == pytest.approx(go, rel=1e-9)
    assert l == pytest.approx(lo, rel=1e-10)


@pytest.mark.parametrize("bad", [dict(G=0.0), dict(G=float("nan")), dict(rho0=0.0), dict(rho0=-1.0)])
def test_create_rejects_bad_psi_exp_params(lib, bad):
    import ctypes
    p = lbm.Params(nx=16, ny=16, eos="psi_exp", G=-2.0, rho0=1.0)
    for k, v in bad.items():
        setattr(p, k, v)
    c = p.c()
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(c), ctypes.byref(h)) == lbm.E_INVALID
    assert h.value is None


def test_psi_exp_above_critical_strength_has_no_loop(lib):
    # G_c = -4 rho0 / 3 for Eq. 5
    with pytest.raises(lbm.LBMError):
        lbm.maxwell(lbm.Params(nx=1, ny=1, eos="psi_exp", G=-1.3, rho0=1.0))
