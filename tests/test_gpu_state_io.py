"""GPU tests of saved lattice states (lbm_save / lbm_load, include/lbm.h):
a run saved half way and resumed in a fresh context repeats the uninterrupted
run bit for bit (the single-pass FP32 kernel, whose saved stencil field the
resumed step reads, and the two-pass FP64 path); a state loads into a context
at another temperature; files that are not states, truncated or corrupted,
and size or precision mismatches are refused without touching the context."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

CS = inputs.EOS_TABLE["cs"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()


def params(nx, ny, prec, Tr=0.8, grad="hdm"):
    return lbm.Params(nx=nx, ny=ny, eos="cs", a=CS["a"], b=CS["b"], Tr=Tr, k=CS["k"], prec=prec, grad=grad)


def droplet(nx, ny):
    op = oracle.params_at(nx, ny, "cs", CS["a"], CS["b"], 0.8, k=CS["k"])
    g, l, _ = oracle.maxwell(op)
    return inputs.droplet(nx, ny, min(nx, ny) / 4, g, l)


@pytest.mark.parametrize("nx,ny,prec,grad", [(128, 96, "f32", "hdm"), (132, 70, "f32", "cdm"), (64, 40, "f64", "hdm")])
def test_resume_repeats_the_uninterrupted_run(tmp_path, nx, ny, prec, grad):
    rho = droplet(nx, ny)
    p = params(nx, ny, prec, grad=grad)
    with lbm.Lattice(p) as lat:
        lat.init_density(rho)
        lat.step(40)
        ref = lat.get_f()
    path = tmp_path / "state.lbm"
    with lbm.Lattice(p) as lat:
        lat.init_density(rho)
        lat.step(17)
        lat.save(path)
        lat.step(5)       # moves on: the file keeps step 17
    with lbm.Lattice(p) as lat:
        lat.load(path)
        lat.step(23)
        got = lat.get_f()
    assert np.array_equal(got, ref)


def test_load_at_another_temperature_and_refusals(tmp_path):
    nx, ny = 128, 64
    rho = droplet(nx, ny)
    path = tmp_path / "s.lbm"
    with lbm.Lattice(params(nx, ny, "f32")) as lat:
        lat.init_density(rho)
        lat.step(5)
        f5 = lat.get_f()
        lat.save(path)
    # another temperature: the state loads, the step forms its own stencil field
    with lbm.Lattice(params(nx, ny, "f32", Tr=0.85)) as lat:
        lat.load(path)
        assert np.array_equal(lat.get_f(), f5)
        lat.step(3)
        assert np.isfinite(lat.get_f()).all()
    # size and precision mismatches
    for q in (params(nx + 4, ny, "f32"), params(nx, ny, "f64")):
        with lbm.Lattice(q) as lat:
            with pytest.raises(lbm.LBMError) as ei:
                lat.load(path)
            assert ei.value.status == lbm.E_INVALID
    # not a state, truncated, corrupted, missing: refused, the context keeps its state
    raw = path.read_bytes()
    bad = {"garbage": b"not a lattice state" * 10, "truncated": raw[: len(raw) // 2],
           "corrupted": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:]}
    with lbm.Lattice(params(nx, ny, "f32")) as lat:
        lat.init_density(rho)
        before = lat.get_f()
        for name, data in bad.items():
            (tmp_path / name).write_bytes(data)
            with pytest.raises(lbm.LBMError) as ei:
                lat.load(tmp_path / name)
            assert ei.value.status == lbm.E_IO, name
        with pytest.raises(lbm.LBMError) as ei:
            lat.load(tmp_path / "missing.lbm")
        assert ei.value.status == lbm.E_IO
        assert np.array_equal(lat.get_f(), before)
        with pytest.raises(lbm.LBMError) as ei:
            lat.save(tmp_path / "no_such_dir" / "x.lbm")
        assert ei.value.status == lbm.E_IO
    # nothing to save before initialisation
    with lbm.Lattice(params(nx, ny, "f32")) as lat:
        with pytest.raises(lbm.LBMError) as ei:
            lat.save(tmp_path / "early.lbm")
        assert ei.value.status == lbm.E_STATE
    assert not os.path.exists(tmp_path / "early.lbm")
