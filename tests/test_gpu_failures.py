"""Failure handling that needs no GPU fault: device-memory exhaustion made on
the host (LBM_DEBUG_FAIL_ALLOC, see lbm_debug_alloc_stats in include/lbm.h).
Every allocation of lbm_create, lbm_batch_create, the host-array staging and
the reverse-mode tape is made to fail in turn; each call answers
LBM_E_NOMEM, frees what it took (the library's live-allocation counts return
to where they were) and leaves the context usable."""
import os

import numpy as np
import pytest

from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu
VAR = "LBM_DEBUG_FAIL_ALLOC"


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()
    yield
    os.environ.pop(VAR, None)


def fail_after(n):
    os.environ[VAR] = str(n)


def no_failures():
    os.environ.pop(VAR, None)


def cs(nx, ny, prec="f32"):
    t = inputs.EOS_TABLE["cs"]
    return lbm.Params(nx=nx, ny=ny, eos="cs", a=t["a"], b=t["b"], Tr=0.8, k=t["k"], prec=prec)


def walk(make, max_allocs=40):
    """Fail allocation n = 0, 1, ... of make() until it succeeds; every
    failure must answer E_NOMEM and leak nothing.  Returns the number of
    allocations make() needs."""
    base = lbm.alloc_stats()
    for n in range(max_allocs):
        fail_after(n)
        try:
            obj = make()
        except lbm.LBMError as e:
            no_failures()
            assert e.status == lbm.E_NOMEM, (n, e)
            assert lbm.alloc_stats() == base, n
            continue
        no_failures()
        obj.close()
        assert lbm.alloc_stats() == base
        return n
    raise AssertionError("never succeeded")


@pytest.mark.parametrize("nx,ny,prec", [(128, 128, "f32"), (64, 40, "f32"), (48, 48, "f64")])
def test_create_fails_cleanly_at_every_allocation(nx, ny, prec):
    n = walk(lambda: lbm.Lattice(cs(nx, ny, prec)))
    assert n >= 6      # f twice, the potential field(s), reduction scratch, observables, error word


def test_batch_create_fails_cleanly_at_every_allocation():
    ps = [cs(256, 8), cs(96, 40), cs(64, 64)]
    n = walk(lambda: lbm.Batch(ps))
    assert n >= 9


def test_staging_and_tape_allocations_fail_cleanly():
    torch = pytest.importorskip("torch")
    p = cs(128, 128)
    g, l = lbm.maxwell(p)
    rho0 = inputs.droplet(128, 128, 30, g, l)
    with lbm.Lattice(p) as lat:
        base = lbm.alloc_stats()
        fail_after(0)                          # the host-array staging of init_density
        with pytest.raises(lbm.LBMError) as ei:
            lat.init_density(rho0)
        no_failures()
        assert ei.value.status == lbm.E_NOMEM and lbm.alloc_stats() == base
        lat.init_density(rho0)                 # usable afterwards
        lat.step(5)
        r_ok, _, _ = lat.moments()
        x = torch.tensor(rho0, dtype=torch.float32, device="cuda")
        rT = torch.empty_like(x)
        base = lbm.alloc_stats()
        for n in (0, 3, 20):                   # checkpoints, then the reverse-sweep buffers
            fail_after(n)
            with pytest.raises(lbm.LBMError) as ei:
                lat.adjoint_forward(x.data_ptr(), 100, 10, rT.data_ptr())
            no_failures()
            assert ei.value.status == lbm.E_NOMEM
            assert lbm.alloc_stats() == base, n
        lat.adjoint_forward(x.data_ptr(), 100, 10, rT.data_ptr())
        lat.sync()
        assert np.isfinite(rT.cpu().numpy()).all()
