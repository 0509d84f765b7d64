"""The bounds-checked build (-DLBM_CHECKED, lbm_debug_check_canaries in
include/lbm.h): every kernel checks the indices of its global and
distributed-shared-memory accesses and reports one outside its buffer in the
error word instead of making it, and every device allocation carries a canary
past its end.  The small and degenerate lattices (8 x 8, 3 x 5, 1 x 16,
200 x 1, lines shorter than the stencil), ragged single-pass strips, walls,
the single-pass CDM variant, the batch in its grid, cluster and grouped
forms, the allocation-free step, the gradient entry point and the reverse
mode (single-pass records and plain rows) run through it in a child process
(the checked library is the one that process loads); each answers without a
bounds report, matches the FP64 oracle at the usual bars (the reverse mode:
a finite gradient), and leaves every canary intact.  The host arrays go in
place or through staging as the device allows.  No access is made outside
a buffer and no GPU fault is provoked: a failed check skips the access."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent('''
    import numpy as np
    import torch
    import oracle
    from paper_1712_06079_gb300 import inputs, lbm
    lbm.load()
    assert lbm.damaged_canaries() == 0                 # the checked library is loaded
    EOS = inputs.EOS_TABLE

    def case(nx, ny, eos, Tr, force, grad, prec, walls=False, steps=3):
        t = EOS[eos]
        gp = lbm.Params(nx=nx, ny=ny, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=Tr, k=t["k"],
                        force=force, grad=grad, prec=prec, walls=walls)
        op = oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=t["k"], force=force,
                              grad=grad, walls=walls)
        g, l, _ = oracle.maxwell(op)
        rho = inputs.droplet(nx, ny, min(nx, ny) / 4, g, l) if min(nx, ny) > 8 else inputs.slab(nx, ny, g, l)
        with lbm.Lattice(gp) as lat:
            lat.init_density(rho)
            lat.step(steps)
            r, _, _ = lat.moments()                    # synchronising: a bounds report raises here
        ro, _, _ = oracle.moments(op, oracle.run(op, oracle.init(op, rho), steps))
        err = float(np.max(np.abs(r - ro) / ro))
        assert err < (1e-12 if prec == "f64" else 1e-5), (nx, ny, prec, err)

    for prec in ("f64", "f32"):
        case(8, 8, "cs", 0.8, "sc", "hdm", prec)
        case(3, 5, "vdw", 0.8, "zc", "hdm", prec)
        case(1, 16, "cs", 0.8, "sc", "hdm", prec)
        case(200, 1, "pr", 0.8, "sc", "hdm", prec)
        case(16, 8, "rk", 0.8, "zc", "cdm", prec)
        case(40, 8, "cs", 0.8, "zc", "hdm", prec, walls=True)
    case(132, 129, "cs", 0.8, "sc", "hdm", "f32")              # single-pass, ragged strip
    case(256, 72, "pr", 0.8, "zc", "hdm", "f32", walls=True)   # single-pass with walls
    case(132, 70, "vdw", 0.85, "sc", "cdm", "f32")             # single-pass, CDM variant
    case(132, 70, "vdw", 0.85, "zc", "cdm", "f32", walls=True)
    # the batch, grid and cluster forms (uneven slices)
    ps = []
    for nx, eos in ((257, "pr"), (331, "cs"), (613, "rk")):
        t = EOS[eos]
        ps.append(lbm.Params(nx=nx, ny=8, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=0.8, k=t["k"], prec="f32"))
    rho0 = [inputs.slab(p.nx, 8, *lbm.maxwell(p)) for p in ps]
    outs = []
    for c in (0, 4, -1):
        with lbm.Batch(ps) as b:
            if c > 0:
                b.set_cluster(c, 256)
            if c < 0:
                b.set_groups(0, 256)
            b.init_density(rho0)
            b.step(5)
            outs.append(b.density())
    for other in outs[1:]:
        for u, v in zip(outs[0], other):
            assert np.array_equal(u, v)
    # the allocation-free step and the gradient entry point
    t = EOS["cs"]
    p = lbm.Params(nx=48, ny=40, eos="cs", a=t["a"], b=t["b"], Tr=0.8, k=t["k"], prec="f32")
    f0 = torch.tensor(oracle.init(oracle.params_at(48, 40, "cs", t["a"], t["b"], 0.8, k=t["k"]),
                                  np.full((40, 48), 0.2)), dtype=torch.float32, device="cuda")
    f1 = torch.empty_like(f0)
    torch.cuda.synchronize()
    assert lbm.step_noalloc(p, f0.data_ptr(), f1.data_ptr()) == lbm.OK
    with lbm.Lattice(p) as lat:
        lat.gradient(inputs.uniform01(5, 48 * 40).reshape(40, 48), 1.0)
    # the reverse mode: single-pass records (FP32, tau 1 and tau 0.8), plain rows (FP64, CDM)
    from paper_1712_06079_gb300.autograd import rollout
    for nx, ny, prec, grad, tau in ((64, 64, "f32", "hdm", 1.0), (100, 70, "f32", "hdm", 0.8),
                                    (40, 36, "f64", "hdm", 1.0), (48, 40, "f32", "cdm", 1.2)):
        pa = lbm.Params(nx=nx, ny=ny, eos="cs", a=t["a"], b=t["b"], Tr=0.8, k=t["k"], tau=tau, grad=grad, prec=prec,
                        stream=torch.cuda.current_stream().cuda_stream)
        g, l = lbm.maxwell(pa)
        dt = torch.float64 if prec == "f64" else torch.float32
        with lbm.Lattice(pa) as lat:
            r0 = torch.tensor(inputs.droplet(nx, ny, min(nx, ny) / 4, g, l), dtype=dt, device="cuda",
                              requires_grad=True)
            Tr = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
            G = torch.tensor(-1.0, dtype=torch.float64, requires_grad=True)
            rT = rollout(lat, r0, Tr, G, 20, 5)
            (rT.double() ** 2).sum().backward()
            assert torch.isfinite(r0.grad).all() and np.isfinite(float(Tr.grad))
            lat.sync()
    assert lbm.damaged_canaries() == 0
    print("checked build ok")
''')


def test_checked_build_runs_clean():
    from paper_1712_06079_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, LBM_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
