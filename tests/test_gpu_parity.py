"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs.

Bars: FP64 path within 1e-12 relative per step (element by element over all
nine populations); FP32 path within 1e-5 relative on rho, cell by cell, after
1000 steps of the relaxing droplet and flat-interface workloads; observables in
FP64."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

EOS = dict(inputs.EOS_TABLE)
EOS["rks"] = dict(a=9 / 49, b=2 / 21, omega=0.344, k=0.01)  # Soave-Redlich-Kwong, water


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()


def make(nx, ny, eos="cs", Tr=0.8, force="sc", grad="hdm", tau=1.0, prec="f64", k=None, radius=0):
    t = EOS[eos]
    kk = t["k"] if k is None else k
    gp = lbm.Params(nx=nx, ny=ny, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=Tr, k=kk, tau=tau,
                    force=force, grad=grad, prec=prec, hdm_radius=radius)
    op = oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=kk, tau=tau, force=force, grad=grad)
    return gp, op


def perturbed_state(op, rho, seed):
    # f^eq(rho, u) with a small seeded velocity and an off-equilibrium part
    ny, nx = rho.shape
    xi = inputs.uniform01(seed, 11 * nx * ny).reshape(11, ny, nx)
    ux, uy = 0.02 * (xi[0] - 0.5), 0.02 * (xi[1] - 0.5)
    f = oracle.init(op, rho, ux, uy)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    return f * (1.0 + 1e-3 * (xi[2:] - 0.5) * w / w.max())


CASES_F64 = [
    # (nx, ny, eos, Tr, force, grad, tau)
    (128, 128, "cs", 0.8, "sc", "hdm", 1.0),    # droplet workload
    (1024, 8, "pr", 0.7, "zc", "hdm", 1.0),     # flat interface, folded y stencil
    (1024, 8, "pr", 0.7, "zc", "cdm", 1.0),
    (96, 40, "vdw", 0.9, "sc", "cdm", 0.8),
    (37, 23, "rk", 0.75, "zc", "hdm", 1.3),     # ragged tiles, odd sizes
    (8, 8, "cs", 0.8, "sc", "hdm", 1.0),        # smaller than the stencil
    (3, 5, "vdw", 0.8, "zc", "hdm", 1.0),
    (1, 16, "cs", 0.8, "sc", "hdm", 1.0),       # degenerate axis: d/dx = 0
    (200, 1, "pr", 0.8, "sc", "hdm", 1.0),
    (70, 90, "rks", 0.8, "sc", "hdm", 1.0),
]


@pytest.mark.parametrize("nx,ny,eos,Tr,force,grad,tau", CASES_F64)
def test_f64_one_step_parity(nx, ny, eos, Tr, force, grad, tau):
    gp, op = make(nx, ny, eos, Tr, force, grad, tau)
    g, l, _ = oracle.maxwell(op)
    rho = inputs.droplet(nx, ny, min(nx, ny) / 4, g, l) if min(nx, ny) > 8 else inputs.slab(nx, ny, g, l)
    f0 = perturbed_state(op, rho, seed=nx * 1000 + ny)
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        lat.step(1)
        fg = lat.get_f()
    fo = oracle.step(op, f0)
    rel = np.abs(fg - fo) / np.abs(fo)
    assert rel.max() < 1e-12, rel.max()


def test_f64_moments_and_observables_parity():
    gp, op = make(128, 96, "cs", 0.8, "sc", "hdm")
    g, l, _ = oracle.maxwell(op)
    f0 = perturbed_state(op, inputs.droplet(128, 96, 25, g, l), seed=5)
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        r, vx, vy = lat.moments()
        obs = lat.observables()
    ro, vxo, vyo = oracle.moments(op, f0)
    assert np.allclose(r, ro, rtol=1e-13, atol=0)
    scale = np.abs(vxo).max()
    assert np.abs(vx - vxo).max() < 1e-12 * scale and np.abs(vy - vyo).max() < 1e-12 * scale
    assert obs["mass"] == pytest.approx(ro.sum(), rel=1e-13)
    assert obs["mom_x"] == pytest.approx((ro * vxo).sum(), abs=1e-12 * ro.sum() * scale)
    assert obs["max_speed"] == pytest.approx(np.sqrt(vxo ** 2 + vyo ** 2).max(), rel=1e-12)
    assert obs["rho_min"] == pytest.approx(ro.min(), rel=1e-14)
    assert obs["rho_max"] == pytest.approx(ro.max(), rel=1e-14)


def test_f64_droplet_2000_steps():
    # workload: 128^2 CS Tr=0.8 droplet R=30, SC + HDM, tau = 1, 2000 steps
    gp, op = make(128, 128, "cs", 0.8, "sc", "hdm")
    g, l, _ = oracle.maxwell(op)
    rho0 = inputs.droplet(128, 128, 30, g, l)
    with lbm.Lattice(gp) as lat:
        lat.init_density(rho0)
        lat.step(2000)
        r, vx, vy = lat.moments()
        obs = lat.observables()
    fo = oracle.run(op, oracle.init(op, rho0), 2000)
    ro, vxo, vyo = oracle.moments(op, fo)
    assert np.abs(r - ro).max() / ro.max() < 1e-10
    assert np.sqrt(vx ** 2 + vy ** 2).max() == pytest.approx(np.sqrt(vxo ** 2 + vyo ** 2).max(), rel=1e-7)
    # mass is conserved to FP64 rounding accumulated over 2000 steps
    assert abs(obs["mass"] - rho0.sum()) / rho0.sum() < 2e-12
    assert abs(obs["mass"] - ro.sum()) / ro.sum() < 2e-12


def bulk_means(rho, case):
    ny, nx = rho.shape
    if case == "droplet":   # 5 x 5 centre of the drop, 5 x 5 block at the corner (vapour)
        liq = rho[ny // 2 - 2: ny // 2 + 3, nx // 2 - 2: nx // 2 + 3].mean()
        gas = np.roll(np.roll(rho, 2, 0), 2, 1)[:5, :5].mean()
    else:                   # slab centre and vapour centre, +-nx/16, averaged over y
        prof = rho.mean(0)
        liq = prof[nx // 2 - nx // 16: nx // 2 + nx // 16 + 1].mean()
        gas = np.r_[prof[: nx // 16 + 1], prof[-nx // 16:]].mean()
    return liq, gas


def golden_fp32_limits():
    # pointwise error after 1000 steps of the oracle's step restated with FP32
    # storage and FP32 or FP64 arithmetic (tests/golden/make_fp32_limits.py)
    rows = {}
    for line in open(os.path.join(HERE, "golden", "fp32_restatement_errors.txt")):
        if line.strip() and not line.startswith("#"):
            case, arith, store, err = line.split()
            rows[(case, arith)] = float(err)
    return rows


@pytest.mark.parametrize("case,two_pass", [("droplet", False), ("droplet", True), ("slab", False)])
def test_f32_1000_steps_against_f64_oracle(case, two_pass):
    # FP32 production path vs the FP64 oracle after 1000 steps, bar
    # max_x |rho32 - rho64| / |rho64| < 1e-5.  The droplet runs the single-pass
    # FP32 kernel (FP32 arithmetic) by default and the two-pass kernels with
    # LBM_FLAG_TWO_PASS; the slab (ny = 8) always runs the two-pass kernels,
    # which compute FP32 lattices in FP64 arithmetic: a plain FP32 evaluation
    # of the step misses the bar on the slab by 30x (tests/test_oracle_fp32.py).
    # Every reported observable's FP32 error is printed.
    if case == "droplet":   # 128^2 CS Tr=0.8 droplet R=30, SC + HDM
        gp, op = make(128, 128, "cs", 0.8, "sc", "hdm", prec="f32")
        g, l, _ = oracle.maxwell(op)
        rho0 = inputs.droplet(128, 128, 30, g, l)
    else:                   # 1024 x 8 PR Tr=0.7 flat slab, ZC + HDM
        gp, op = make(1024, 8, "pr", 0.7, "zc", "hdm", prec="f32")
        g, l, _ = oracle.maxwell(op)
        rho0 = inputs.slab(1024, 8, g, l)
    gp.two_pass = two_pass
    with lbm.Lattice(gp) as lat:
        lat.init_density(rho0)
        lat.set_timing(True)
        lat.step(1000)
        kinds = set(lat.timing()["kernels"])
        r, vx, vy = lat.moments()
        obs = lat.observables()
    assert ("fused_step" in kinds) == (case == "droplet" and not two_pass)
    ro, vxo, vyo = oracle.moments(op, oracle.run(op, oracle.init(op, rho0), 1000))
    pointwise = float(np.max(np.abs(r - ro) / np.abs(ro)))
    normwise = float(np.max(np.abs(r - ro)) / np.max(np.abs(ro)))
    liq32, gas32 = bulk_means(r, case)
    liq64, gas64 = bulk_means(ro, case)
    speed32, speed64 = np.hypot(vx, vy).max(), np.hypot(vxo, vyo).max()
    errs = {"rho pointwise": pointwise, "rho normwise": normwise, "rho_l": liq32 / liq64 - 1,
            "rho_g": gas32 / gas64 - 1, "ratio": (liq32 / gas32) / (liq64 / gas64) - 1,
            "mass": obs["mass"] / ro.sum() - 1, "max|v|": speed32 / speed64 - 1}
    print(f"FP32 vs FP64 oracle, {case}, two_pass={two_pass}: " +
          ", ".join(f"{k} {v:+.2e}" for k, v in errs.items()))
    assert pointwise < 1e-5, pointwise
    assert abs(errs["rho_l"]) < 1e-5 and abs(errs["rho_g"]) < 1e-5 and abs(errs["mass"]) < 1e-6
    assert abs(errs["max|v|"]) < 1e-3
    # and well inside what a plain FP32 evaluation of the oracle's step reaches
    assert pointwise < golden_fp32_limits()[(case, "f32")] / 2


def test_f32_one_step_full_size_spinodal():
    # the throughput workload at full size: 4096^2 CS Tr=0.7, mean of the
    # coexistence pair with 1 % relative noise; one step against the oracle,
    # with the default segment height and with the tuned one the benchmark runs
    n = 4096
    gp, op = make(n, n, "cs", 0.7, "sc", "hdm", prec="f32")
    rho0 = inputs.spinodal(n, n, inputs.CS_TR07_MEAN)
    oracle.set_threads(oracle.max_threads())
    ro, vxo, _ = oracle.moments(op, oracle.step(op, oracle.init(op, rho0)))
    with lbm.Lattice(gp) as lat:
        for tuned in (False, True):
            lat.init_density(rho0)
            if tuned:
                assert lat.tune_segment_rows() > 0
            lat.step(1)
            r, vx, _ = lat.moments()
            assert np.max(np.abs(r - ro) / ro) < 2e-6
            # v carries the FP32 HDM gradient of a 1 %-noise field: cancellation in the
            # stencil leaves ~1e-5 of the largest velocity
            assert np.max(np.abs(vx - vxo)) < 1e-4 * np.abs(vxo).max()


def test_f32_full_size_benchmark_run_properties():
    # the benchmark's run: 4096^2 spinodal, tuned launch, 2000 steps, checked
    # by what holds at any size (the oracle cannot follow 2000 steps of 16.8 M
    # cells): mass conserved to FP32 rounding, the density finite and positive,
    # and the spinodal state separated into vapour and liquid near the Maxwell
    # pair (9.3e-3, 0.358), as the oracle's 256^2 run of the same recipe does
    n = 4096
    gp, op = make(n, n, "cs", 0.7, "sc", "hdm", prec="f32")
    rho0 = inputs.spinodal(n, n, inputs.CS_TR07_MEAN)
    m0 = float(rho0.astype(np.float32).astype(np.float64).sum())
    with lbm.Lattice(gp) as lat:
        lat.init_density(rho0)
        assert lat.tune_segment_rows() > 0
        lat.step(2000)
        obs = lat.observables()
    assert abs(obs["mass"] - m0) / m0 < 1e-6
    assert 0 < obs["rho_min"] < 0.03 and 0.3 < obs["rho_max"] < 0.45
    assert np.isfinite(obs["max_speed"]) and obs["max_speed"] < 0.2


def test_unstable_state_is_reported_and_cleared():
    gp, op = make(32, 32, "cs", 0.8, "sc", "hdm")
    f = oracle.init(op, np.full((32, 32), 0.1))
    f[:, 5, 7] = -0.01  # negative density at one cell
    with lbm.Lattice(gp) as lat:
        lat.set_f(f)
        lat.step(1)
        with pytest.raises(lbm.LBMError) as ei:
            lat.sync()
        assert ei.value.status == lbm.E_UNSTABLE
        with pytest.raises(lbm.LBMError):
            lat.step(1)
        lat.init_density(np.full((32, 32), 0.1))
        lat.step(3)
        lat.sync()


def test_step_before_init_is_rejected():
    gp, _ = make(16, 16)
    with lbm.Lattice(gp) as lat:
        with pytest.raises(lbm.LBMError) as ei:
            lat.step(1)
        assert ei.value.status == lbm.E_STATE


FUSED_CASES = [
    # (nx, ny, eos, Tr, force, grad): strips of 120 columns, segments of 128 rows, ragged edges
    (132, 129, "cs", 0.8, "sc", "hdm"),
    (64, 54, "vdw", 0.85, "zc", "hdm"),   # smallest lattice the single-pass kernel takes
    (256, 200, "pr", 0.75, "sc", "hdm"),
    (4096, 64, "rk", 0.8, "zc", "hdm"),
    (132, 129, "vdw", 0.85, "sc", "cdm"),   # the kernel's CDM variant (Eq. 15)
    (256, 64, "pr", 0.9, "zc", "cdm"),   # (ZC + CDM at T/Tc 0.8 blows up within 20 steps, in the oracle too)
]


def run_f32(gp, f0, steps, two_pass):
    gp.two_pass = two_pass
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        lat.set_timing(True)
        lat.step(steps)
        kinds = set(lat.timing()["kernels"])
        fg = lat.get_f()
    return fg, kinds


@pytest.mark.parametrize("nx,ny,eos,Tr,force,grad", FUSED_CASES)
def test_f32_single_pass_kernel_parity(nx, ny, eos, Tr, force, grad):
    # the single-pass FP32 kernel against the FP64 oracle (one step, all
    # populations) and against the two-pass FP32 kernels (20 steps)
    gp, op = make(nx, ny, eos, Tr, force, grad, prec="f32")
    g, l, _ = oracle.maxwell(op)
    f0 = perturbed_state(op, inputs.droplet(nx, ny, min(nx, ny) / 4, g, l), seed=nx + 7 * ny)
    f1, kinds = run_f32(gp, f0, 1, two_pass=False)
    assert "fused_step" in kinds and "collide" not in kinds
    fo = oracle.step(op, f0)
    # one FP32 step vs FP64: a few ulps per population (more where U = k p - rho/3
    # cancels, at liquid densities of PR)
    assert np.max(np.abs(f1 - fo) / fo) < 1e-5
    fa, kinds_a = run_f32(gp, f0, 20, two_pass=False)
    fb, kinds_b = run_f32(gp, f0, 20, two_pass=True)
    assert "collide" in kinds_b and "fused_step" not in kinds_b
    assert np.max(np.abs(fa - fb) / np.abs(fb)) < 1e-5


def test_f32_arith_flag_keeps_fp32_arithmetic_in_the_two_pass_kernels():
    # LBM_FLAG_F32_ARITH: the two-pass kernels compute an FP32 lattice in FP32.
    # One step against the oracle's step of the same FP32-rounded state: the
    # default (FP64 arithmetic on FP32 storage) differs by the rounding of the
    # result to FP32 alone; FP32 arithmetic by a few ulp more (PR, where
    # U = k p - rho/3 nearly cancels at liquid density)
    gp, op = make(96, 40, "pr", 0.75, "zc", "hdm", prec="f32")
    g, l, _ = oracle.maxwell(op)
    f0 = perturbed_state(op, inputs.droplet(96, 40, 12, g, l), seed=77)
    f0 = f0.astype(np.float32).astype(np.float64)
    fo = oracle.step(op, f0)
    outs = []
    for flag, bar in ((False, 1.2e-7), (True, 5e-5)):
        gp.f32_arith = flag
        with lbm.Lattice(gp) as lat:
            lat.set_f(f0)
            lat.step(1)
            outs.append(lat.get_f())
        err = np.max(np.abs(outs[-1] - fo) / fo)
        print(f"f32_arith={flag}: one step {err:.2e}")
        assert err < bar, (flag, err)
    d = np.max(np.abs(outs[0] - outs[1]) / outs[0])
    assert 0 < d < 5e-5, d


def test_f32_single_pass_segment_height_does_not_change_results():
    # the CTA segment height is a launch shape: every cell takes the same
    # arithmetic except the d/dy forward recurrence, which carries its sum
    # from the segment's first row (terms beyond the 26-row stencil radius,
    # weight r^26 ~ 1e-11) and so rounds along a different path; the states
    # agree to the bar the single-pass and two-pass FP32 paths are held to
    nx, ny = 252, 200
    gp, op = make(nx, ny, "cs", 0.8, "sc", "hdm", prec="f32")
    g, l, _ = oracle.maxwell(op)
    f0 = perturbed_state(op, inputs.droplet(nx, ny, 50, g, l), seed=3)
    outs = {}
    for rows in (0, 1, 6, 7, 9, 14, 62, 126, 128, 200):
        with lbm.Lattice(gp) as lat:
            lat.set_segment_rows(rows)
            used = lat.segment_rows()
            assert used == rows or (rows == 0 and used > 0)
            lat.set_f(f0)
            lat.step(12)
            outs[rows] = lat.get_f()
    for rows, fr in outs.items():
        assert np.max(np.abs(fr - outs[0]) / np.abs(outs[0])) < 1e-5, rows
    with lbm.Lattice(gp) as lat:
        for bad in (-1, ny + 1):
            with pytest.raises(lbm.LBMError) as ei:
                lat.set_segment_rows(bad)
            assert ei.value.status == lbm.E_INVALID
    gp.two_pass = True
    with lbm.Lattice(gp) as lat:
        assert lat.segment_rows() == 0


def test_f32_segment_height_tuner_keeps_state():
    # the tuner times trial launches on the current state: it leaves the
    # state it found, keeps a whole-slab height 8k - 2 <= ny, and the steps
    # after it are bit-identical to steps with that height set by hand
    nx, ny = 252, 200
    gp, op = make(nx, ny, "cs", 0.8, "sc", "hdm", prec="f32")
    g, l, _ = oracle.maxwell(op)
    f0 = perturbed_state(op, inputs.droplet(nx, ny, 50, g, l), seed=3)
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        lat.step(3)
        before = lat.get_f()
        rows = lat.tune_segment_rows(2)
        assert rows % 8 == 6 and 6 <= rows <= ny
        assert lat.segment_rows() == rows
        assert np.array_equal(lat.get_f(), before)
        lat.step(5)
        tuned = lat.get_f()
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        lat.step(3)
        lat.set_segment_rows(rows)
        lat.step(5)
        assert np.array_equal(lat.get_f(), tuned)
    with lbm.Lattice(gp) as lat:
        with pytest.raises(lbm.LBMError) as ei:
            lat.tune_segment_rows(2)
        assert ei.value.status == lbm.E_STATE
        lat.set_f(f0)
        for bad in (0, 1001):
            with pytest.raises(lbm.LBMError) as ei:
                lat.tune_segment_rows(bad)
            assert ei.value.status == lbm.E_INVALID
    gp.two_pass = True
    with lbm.Lattice(gp) as lat:
        lat.set_f(f0)
        assert lat.tune_segment_rows(2) == 0


def test_f32_single_pass_is_deterministic():
    # the same input stepped twice in fresh contexts gives bit-identical
    # states: every value the kernel reads from shared memory has landed (the
    # bulk copies complete on mbarriers) and every output is written once.
    # A spinodal lattice amplifies any difference step by step.
    n = 512
    gp, op = make(n, n, "cs", 0.7, "sc", "hdm", prec="f32")
    rho0 = inputs.spinodal(n, n, inputs.CS_TR07_MEAN, seed=9)
    outs = []
    for _ in range(3):
        with lbm.Lattice(gp) as lat:
            lat.init_density(rho0)
            lat.step(300)
            outs.append(lat.get_f())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_host_arrays_in_place_equal_staged(prec):
    # Where the device accesses pageable host memory in place (Grace with
    # NVLink-C2C), lbm_init_density reads the caller's FP64 arrays directly and
    # lbm_moments writes arrays whose pages are all resident directly;
    # LBM_FLAG_STAGED_HOST keeps the pinned staging path.  All give the same
    # values; an invalid rho is reported at its lowest index and leaves the
    # state as it was.
    nx, ny = 200, 136
    gp, op = make(nx, ny, "pr", 0.75, "zc", "hdm", prec=prec)
    g, l, _ = oracle.maxwell(op)
    rho = inputs.droplet(nx, ny, 30, g, l)
    xi = inputs.uniform01(77, 2 * nx * ny).reshape(2, ny, nx)
    ux, uy = 0.01 * (xi[0] - 0.5), 0.01 * (xi[1] - 0.5)
    bad = rho.copy()
    bad[9, 3] = np.nan
    bad[3, 7] = -1.0   # the lowest bad index: 3 * nx + 7
    outs = []
    for staged in (False, True):
        gp.staged_host = staged
        with lbm.Lattice(gp) as lat:
            if staged:
                assert not lat.host_in_place()
            lat.init_density(rho, ux, uy)
            lat.step(5)
            m1 = lat.moments()                         # fresh arrays: through the staging buffer
            resident = tuple(np.full((ny, nx), -1.0) for _ in range(3))
            m1b = lat.moments(out=resident)            # resident arrays: written in place where possible
            for a, b in zip(m1, m1b):
                assert np.array_equal(a, b)
            with pytest.raises(lbm.LBMError) as ei:
                lat.init_density(bad)
            assert ei.value.status == lbm.E_INVALID and f"rho[{3 * nx + 7}]" in str(ei.value)
            m2 = lat.moments()
            for a, b in zip(m1, m2):
                assert np.array_equal(a, b)
            outs.append(m1)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_f32_cdm_single_pass_1000_steps_no_worse_than_plain_fp32():
    # The CDM (comparison arm, Eq. 15) in the single-pass kernel, 1000 steps of
    # the 128^2 CS droplet against the FP64 oracle.  The 1e-5 contract bar is
    # the production HDM path's; for the CDM variant the bar is what the
    # oracle's step restated in plain FP32 arithmetic reaches on the same
    # state (2.8e-5; the kernel: 1.2e-5), and the two-pass path (FP64
    # arithmetic on FP32 storage) holds 1e-5.
    from oracle.fp32_restatement import Restatement
    gp, op = make(128, 128, "cs", 0.8, "sc", "cdm", prec="f32")
    g, l, _ = oracle.maxwell(op)
    rho = inputs.droplet(128, 128, 30, g, l)
    f0 = oracle.init(op, rho)
    ro = oracle.run(op, f0, 1000).sum(0)
    e_plain = np.max(np.abs(Restatement(op, np.float32, np.float32).run(f0, 1000).sum(0) - ro) / ro)
    errs = {}
    for two_pass in (False, True):
        gp.two_pass = two_pass
        with lbm.Lattice(gp) as lat:
            lat.init_density(rho)
            lat.set_timing(True)
            lat.step(1000)
            kinds = set(lat.timing()["kernels"])
            r = lat.moments()[0]
        assert ("fused_step" in kinds) == (not two_pass)
        errs[two_pass] = float(np.max(np.abs(r - ro) / ro))
    print(f"CDM droplet 1000 steps: single-pass {errs[False]:.2e}, two-pass {errs[True]:.2e}, "
          f"plain FP32 restatement {e_plain:.2e}")
    assert errs[False] < e_plain
    assert errs[True] < 1e-5
