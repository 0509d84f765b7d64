"""lbm_step_noalloc: the step for callers that cannot call cudaMalloc.

Its scratch (the potential field and the error word) is a fixed file-scope
device array, so the caller only passes its own f_in and f_out device buffers.
These tests call it through the C ABI twice in a row and compare each result
with the context-based entry points (lbm_set_f + lbm_step + lbm_get_f) on the
same state, within the tolerances of the other parity tests.  The file is
named to be collected last so that a first-failure run has already run every
other test.
"""
import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()
    return torch


def state(nx, ny, eos, Tr):
    t = inputs.EOS_TABLE[eos]
    op = oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=t["k"])
    g, l, _ = oracle.maxwell(op)
    rho = inputs.droplet(nx, ny, min(nx, ny) / 4, g, l)
    xi = inputs.uniform01(nx * 31 + ny, 2 * nx * ny).reshape(2, ny, nx)
    return oracle.init(op, rho, 0.01 * (xi[0] - 0.5), 0.01 * (xi[1] - 0.5)), t


@pytest.mark.parametrize("prec,nx,ny,eos,tol,walls", [("f64", 96, 80, "cs", 1e-12, False),
                                                     ("f32", 200, 136, "pr", 1e-6, False),
                                                     ("f64", 64, 40, "cs", 1e-12, True)])
def test_noalloc_matches_context_two_calls(torch_cuda, prec, nx, ny, eos, tol, walls):
    torch = torch_cuda
    f0, t = state(nx, ny, eos, 0.8)
    dt = torch.float64 if prec == "f64" else torch.float32
    stream = torch.cuda.current_stream()
    params = lbm.Params(nx=nx, ny=ny, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=0.8, k=t["k"],
                        prec=prec, two_pass=True, walls=walls, stream=stream.cuda_stream)
    # reference: the context path (same two-pass kernels)
    with lbm.Lattice(params) as lat:
        lat.set_f(f0)
        lat.step(1)
        ref1 = lat.get_f()
        lat.step(1)
        ref2 = lat.get_f()
    # caller-owned device buffers (allocated by the test, not by the entry point)
    fa = torch.tensor(f0, dtype=dt, device="cuda").contiguous()
    fb = torch.empty_like(fa)
    fc = torch.empty_like(fa)
    torch.cuda.synchronize()
    assert lbm.step_noalloc(params, fa.data_ptr(), fb.data_ptr()) == lbm.OK
    assert lbm.step_noalloc(params, fb.data_ptr(), fc.data_ptr()) == lbm.OK
    out1 = fb.double().cpu().numpy()
    out2 = fc.double().cpu().numpy()
    assert np.max(np.abs(out1 - ref1) / np.abs(ref1)) < tol
    assert np.max(np.abs(out2 - ref2) / np.abs(ref2)) < tol
    # and the first call left its input untouched
    assert np.array_equal(fa.double().cpu().numpy(), f0.astype(np.float32 if prec == "f32" else np.float64))


# (4 MiB - 256 B) / 8 B: the FP64 potential field's cells in the 4 MiB array
MAX_CELLS = 524_256


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_size_limit_at_its_boundary(torch_cuda, prec):
    # exactly MAX_CELLS cells (1016 x 516) run and match the context path; one
    # cell more (a 524,257 x 1 line) is refused before any device work
    torch = torch_cuda
    nx, ny = 1016, 516
    assert nx * ny == MAX_CELLS
    f0, t = state(nx, ny, "cs", 0.8)
    dt = torch.float64 if prec == "f64" else torch.float32
    params = lbm.Params(nx=nx, ny=ny, eos="cs", a=t["a"], b=t["b"], Tr=0.8, k=t["k"], prec=prec, two_pass=True,
                        stream=torch.cuda.current_stream().cuda_stream)
    with lbm.Lattice(params) as lat:
        lat.set_f(f0)
        lat.step(1)
        ref = lat.get_f()
    fa = torch.tensor(f0, dtype=dt, device="cuda").contiguous()
    fb = torch.empty_like(fa)
    torch.cuda.synchronize()
    assert lbm.step_noalloc(params, fa.data_ptr(), fb.data_ptr()) == lbm.OK
    assert np.max(np.abs(fb.double().cpu().numpy() - ref) / np.abs(ref)) < (1e-12 if prec == "f64" else 1e-6)
    over = lbm.Params(nx=MAX_CELLS + 1, ny=1, eos="cs", a=t["a"], b=t["b"], Tr=0.8, k=t["k"], prec=prec)
    before = fb.clone()
    assert lbm.step_noalloc(over, fa.data_ptr(), fb.data_ptr()) == lbm.E_INVALID
    torch.cuda.synchronize()
    assert torch.equal(fb, before)


def test_noalloc_rejects_oversize_and_bad_arguments(torch_cuda):
    torch = torch_cuda
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    big = lbm.Params(nx=1024, ny=1025, eos="cs", Tr=0.8, k=0.04, prec="f32")   # 1,049,600 cells > limit
    assert lbm.step_noalloc(big, buf.data_ptr(), buf.data_ptr() + 4) == lbm.E_INVALID
    big64 = lbm.Params(nx=1024, ny=513, eos="cs", Tr=0.8, k=0.04, prec="f64")  # 525,312 cells > limit
    assert lbm.step_noalloc(big64, buf.data_ptr(), buf.data_ptr() + 8) == lbm.E_INVALID
    ok = lbm.Params(nx=4, ny=4, eos="cs", Tr=0.8, k=0.04, prec="f32")
    assert lbm.step_noalloc(ok, buf.data_ptr(), buf.data_ptr()) == lbm.E_INVALID   # in place is refused
    assert lbm.step_noalloc(ok, 0, buf.data_ptr()) == lbm.E_INVALID
