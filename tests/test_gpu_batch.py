"""GPU tests of the batched sweep (lbm_batch_*): one persistent launch over
many uneven lattices, each with its own EOS, temperature, tau, force form and
gradient.  Parity against the FP64 oracle per instance, agreement with the
single-lattice contexts, graph replay, the autotuner, and the bounded grid
barrier (a block that never arrives makes the launch give up with
LBM_E_TIMEOUT, without hanging the GPU)."""
import numpy as np
import pytest

import oracle
from paper_1712_06079_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

EOS = dict(inputs.EOS_TABLE)
EOS["rks"] = dict(a=9 / 49, b=2 / 21, omega=0.344, k=0.01)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_06079_gb300 import build
    build.build()
    lbm.load()


def instance(nx, ny, eos, Tr, tau, force="sc", grad="hdm", prec="f64"):
    t = EOS[eos]
    gp = lbm.Params(nx=nx, ny=ny, eos=eos, a=t["a"], b=t["b"], omega=t["omega"], Tr=Tr, k=t["k"], tau=tau,
                    force=force, grad=grad, prec=prec)
    op = oracle.params_at(nx, ny, eos, t["a"], t["b"], Tr, omega=t["omega"], k=t["k"], tau=tau,
                          force=force, grad=grad)
    return gp, op


MIX = [  # uneven sizes, every EOS, both forces and gradients
    (256, 8, "pr", 0.7, 1.0, "zc", "hdm"),
    (328, 8, "cs", 0.8, 0.9, "sc", "hdm"),
    (96, 40, "vdw", 0.85, 1.1, "sc", "cdm"),
    (512, 8, "rk", 0.75, 1.2, "zc", "hdm"),
    (40, 24, "rks", 0.8, 0.8, "sc", "hdm"),
    (1000, 8, "vdw", 0.9, 1.0, "zc", "cdm"),   # ZC + CDM is unstable at low Tr (physics, not the kernel)
]


def slab_state(op, seed):
    g, l, _ = oracle.maxwell(op)
    rho = inputs.slab(op.nx, op.ny, g, l)
    xi = inputs.uniform01(seed, 2 * op.nx * op.ny).reshape(2, op.ny, op.nx)
    return oracle.init(op, rho, 0.01 * (xi[0] - 0.5), 0.01 * (xi[1] - 0.5))


def test_batch_f64_matches_oracle_per_instance():
    pairs = [instance(*m) for m in MIX]
    f0 = [slab_state(op, k + 1) for k, (_, op) in enumerate(pairs)]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.set_f(f0)
        b.step(1)
        f1 = b.get_f()
        b.step(2)      # a second launch of 2 steps (graph replay from the other buffer)
        f3 = b.get_f()
    for (gp, op), a, g1, g3 in zip(pairs, f0, f1, f3):
        o1 = oracle.step(op, a)
        assert np.max(np.abs(g1 - o1) / np.abs(o1)) < 1e-12, (gp.eos, gp.nx)
        o3 = oracle.run(op, a, 3)
        assert np.max(np.abs(g3 - o3) / np.abs(o3)) < 1e-11, (gp.eos, gp.nx)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_moments_match_oracle_per_instance(prec):
    # lbm_batch_moments: rho (Eq. 3) and the half-step velocity of Eq. 11 of
    # every instance against the oracle's moments of the same state (its own
    # FP64 run of the same steps); FP64 at 1e-12, FP32 at its rounding level
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec=prec) for m in MIX]
    f0 = [slab_state(op, k + 21) for k, (_, op) in enumerate(pairs)]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.set_f(f0)
        b.step(3)
        rho, vx, vy = b.moments()
        dens = b.density()
    # FP32: a few ulp per step, more for PR where U = k p - rho/3 nearly cancels at liquid density
    tol_r, tol_v = (1e-12, 1e-11) if prec == "f64" else (1e-5, 1e-3)
    for (gp, op), a, r, u, v, d in zip(pairs, f0, rho, vx, vy, dens):
        ro, vxo, vyo = oracle.moments(op, oracle.run(op, a, 3))
        assert r.shape == ro.shape == (gp.ny, gp.nx)
        assert np.array_equal(r, d)            # the density entry point's rho
        assert np.max(np.abs(r - ro) / ro) < tol_r, (gp.eos, gp.nx)
        scale = max(np.abs(vxo).max(), np.abs(vyo).max())
        assert np.max(np.abs(u - vxo)) < tol_v * scale and np.max(np.abs(v - vyo)) < tol_v * scale, (gp.eos, gp.nx)
    # vx / vy may be left out
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.set_f(f0)
        flat = np.empty(sum(gp.nx * gp.ny for gp, _ in pairs))
        assert b._lib.lbm_batch_moments(b._h, lbm._dp(flat), None, None) == lbm.OK
        assert np.array_equal(flat[: pairs[0][0].nx * pairs[0][0].ny].reshape(pairs[0][0].ny, pairs[0][0].nx),
                              b.density()[0])


def test_batch_f32_matches_single_lattice_contexts():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in MIX]
    f0 = [slab_state(op, k + 11) for k, (_, op) in enumerate(pairs)]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.set_f(f0)
        b.step(100)
        fb = b.get_f()
    for (gp, _), a, got in zip(pairs, f0, fb):
        gp.two_pass = True
        with lbm.Lattice(gp) as lat:
            lat.set_f(a)
            lat.step(100)
            ref = lat.get_f()
        # the batch computes in FP32, the contexts' two-pass kernels in FP64 on
        # FP32-stored distributions: 100 steps apart by FP32 rounding (largest
        # for PR, where U = k p - rho/3 nearly cancels at liquid density)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 3e-5, (gp.eos, gp.nx)


CLUSTER_MIX = MIX[:4]   # split over 2 (FP32), 4 and 8 (FP32) CTAs per instance


@pytest.mark.parametrize("prec,cluster,threads", [("f64", 4, 256), ("f32", 2, 512), ("f32", 4, 256),
                                                  ("f32", 8, 128), ("f32", 8, 1024)])
def test_cluster_form_equals_grid_form(prec, cluster, threads):
    # the cluster form runs the grid form's per-cell arithmetic on shared
    # memory: the same state after every launch, bit for bit, including graph
    # replays from either buffer
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec=prec) for m in CLUSTER_MIX]
    f0 = [slab_state(op, k + 31) for k, (_, op) in enumerate(pairs)]
    outs = []
    for c in (0, cluster):
        with lbm.Batch([gp for gp, _ in pairs]) as b:
            if c:
                b.set_cluster(c, threads)
                assert b.cluster() == c and b.launch() == (threads, c * len(pairs))
            b.set_f(f0)
            states = []
            for n in (1, 6, 6):
                b.step(n)
                states.append(b.get_f())
            outs.append(states)
    for sg, sc in zip(outs[0], outs[1]):
        for u, v in zip(sg, sc):
            assert np.array_equal(u, v)


def test_full_sweep_in_the_benchmark_launch_equals_grid_form():
    # the 64-lattice sweep at full size in the launch the benchmark times
    # (8 CTAs x 1024 threads per lattice): the same state as the grid form
    params, rho0 = [], []
    for d in inputs.sweep_instances(64):
        gp = lbm.Params(nx=d["nx"], ny=d["ny"], eos=d["eos"], a=d["a"], b=d["b"], omega=d["omega"], Tr=d["Tr"],
                        k=d["k"], tau=d["tau"], force="sc", grad="hdm", prec="f32")
        g, l = lbm.maxwell(gp)
        params.append(gp)
        rho0.append(inputs.slab(d["nx"], d["ny"], g, l))
    out = []
    for c in (0, 8, -1):
        with lbm.Batch(params) as b:
            if c > 0:
                b.set_cluster(c, 1024)
            if c < 0:
                b.set_groups(0, 1024)
                assert len(b.groups()) >= 2
            b.init_density(rho0)
            b.step(50)
            out.append(b.density())
    for k in (1, 2):
        for u, v in zip(out[0], out[k]):
            assert np.array_equal(u, v)


ODD_MIX = [  # widths no cluster size divides: slices of uneven width
    (257, 8, "pr", 0.7, 1.0, "zc", "hdm"),
    (331, 8, "cs", 0.8, 0.9, "sc", "hdm"),
    (1001, 8, "vdw", 0.85, 1.1, "sc", "cdm"),
    (613, 8, "rk", 0.75, 1.2, "zc", "hdm"),
]


@pytest.mark.parametrize("prec,cluster,threads", [("f32", 8, 1024), ("f32", 4, 256), ("f64", 4, 256)])
def test_cluster_form_with_uneven_slices_equals_grid_form(prec, cluster, threads):
    # FP64: HDM radius 40 needs slices of 40 columns, and the 1001-wide lattice's
    # slices of 251 FP64 columns do not fit a block's shared memory
    mix = ODD_MIX if prec == "f32" else [m for m in ODD_MIX if m[0] != 1001]
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec=prec) for m in mix]
    f0 = [slab_state(op, k + 61) for k, (_, op) in enumerate(pairs)]
    outs = []
    for c in (0, cluster):
        with lbm.Batch([gp for gp, _ in pairs]) as b:
            if c:
                b.set_cluster(c, threads)
                assert b.cluster() == c
            b.set_f(f0)
            b.step(7)
            b.step(6)
            outs.append(b.get_f())
    for u, v in zip(*outs):
        assert np.array_equal(u, v)
    if prec == "f64":   # and the oracle's step
        for (gp, op), a, got in zip(pairs, f0, outs[1]):
            ref = oracle.run(op, a, 13)
            assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-11, (gp.eos, gp.nx)


@pytest.mark.parametrize("prec,cap,threads", [("f32", 0, 1024), ("f32", 72 * 1024, 512), ("f64", 0, 256),
                                              ("f32", lbm.GROUPS_BALANCED, 1024)])
def test_grouped_form_equals_grid_form(prec, cap, threads):
    # each lattice on the smallest cluster its slices fit: with the whole opt-in
    # shared memory the FP32 mix runs as a group of 2-CTA clusters and one of
    # 4-CTA clusters, each its own launch on its own stream
    mix = ODD_MIX if prec == "f32" else [m for m in ODD_MIX if m[0] != 1001]
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec=prec) for m in mix]
    f0 = [slab_state(op, k + 71) for k, (_, op) in enumerate(pairs)]
    outs = []
    for grouped in (False, True):
        with lbm.Batch([gp for gp, _ in pairs]) as b:
            if grouped:
                b.set_groups(cap, threads)
                assert b.cluster() == -1
                groups = b.groups()
                assert sum(n for _, n in groups) == len(pairs)
                assert [c for c, _ in groups] == sorted({c for c, _ in groups}, reverse=True)
                if prec == "f32" and cap == 0:
                    assert groups == [(4, 1), (2, 3)]
                assert b.launch() == (threads, sum(c * n for c, n in groups))
            b.set_f(f0)
            b.step(7)
            b.step(6)
            outs.append(b.get_f())
    for u, v in zip(*outs):
        assert np.array_equal(u, v)


def test_grouped_form_refusal_keeps_the_form():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in ODD_MIX]
    big = instance(20000, 8, "cs", 0.8, 1.0, prec="f32")   # slices of 2500 columns exceed shared memory
    with lbm.Batch([gp for gp, _ in pairs] + [big[0]]) as b:
        with pytest.raises(lbm.LBMError) as ei:
            b.set_groups(0, 1024)
        assert ei.value.status == lbm.E_INVALID
        assert b.cluster() == 0 and b.groups() == []
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        for bad in (128, 96):
            with pytest.raises(lbm.LBMError):
                b.set_groups(0, bad)
        b.set_groups(0, 512)
        b.set_cluster(0, 256)   # back to the grid form
        assert b.cluster() == 0 and b.groups() == []


def test_cluster_form_f64_matches_oracle():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f64") for m in CLUSTER_MIX]
    f0 = [slab_state(op, k + 41) for k, (_, op) in enumerate(pairs)]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.set_cluster(4, 256)
        b.set_f(f0)
        b.step(3)
        f3 = b.get_f()
    for (gp, op), a, got in zip(pairs, f0, f3):
        ref = oracle.run(op, a, 3)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12, (gp.eos, gp.nx)


def test_cluster_form_refusals_and_instability():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in MIX]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        for c, t in [(8, 256), (3, 256), (16, 256), (1, 256), (4, 96)]:   # 40 / 8 < the HDM halo; bad sizes
            with pytest.raises(lbm.LBMError) as ei:
                b.set_cluster(c, t)
            assert ei.value.status == lbm.E_INVALID
        assert b.cluster() == 0
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in CLUSTER_MIX]
    f0 = [slab_state(op, k + 51) for k, (_, op) in enumerate(pairs)]
    f0[1][:, 3, 100] = -0.01   # a negative density in the second instance
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.set_cluster(8, 256)
        b.set_f(f0)
        b.step(2)
        with pytest.raises(lbm.LBMError) as ei:
            b.sync()
        assert ei.value.status == lbm.E_UNSTABLE
        b.set_cluster(0, 256)
        assert b.cluster() == 0


def test_cluster_autotuner_keeps_state():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in CLUSTER_MIX]
    rho0 = [inputs.slab(op.nx, op.ny, *oracle.maxwell(op)[:2]) for _, op in pairs]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.init_density(rho0)
        before = b.density()
        threads, grid = b.tune(trial_steps=20)
        assert (threads, grid) == b.launch()
        c = b.cluster()
        assert c in (-1, 0, 2, 4, 8)
        if c > 0:
            assert grid == c * len(pairs)
        if c < 0:
            assert grid == sum(cl * n for cl, n in b.groups())
        assert threads in (128, 256, 512, 1024)
        for x, y in zip(before, b.density()):
            assert np.array_equal(x, y)
        b.step(10)
        b.sync()


def test_batch_graph_replay_and_launch_shapes_agree():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f64") for m in MIX[:4]]
    f0 = [slab_state(op, k + 21) for k, (_, op) in enumerate(pairs)]
    outs = []
    for shape, chunks in [((256, 1), [8]), ((128, 2), [4, 4]), ((512, 1), [2, 6])]:
        with lbm.Batch([gp for gp, _ in pairs]) as b:
            b.set_launch(*shape)
            b.set_f(f0)
            for n in chunks:
                b.step(n)
            outs.append(b.get_f())
    for other in outs[1:]:
        for a, c in zip(outs[0], other):
            assert np.array_equal(a, c)


def test_batch_autotuner_keeps_state_and_picks_a_valid_shape():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in MIX]
    rho0 = [inputs.slab(op.nx, op.ny, *oracle.maxwell(op)[:2]) for _, op in pairs]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.init_density(rho0)
        before = b.density()
        threads, grid = b.tune(trial_steps=20)
        # no single cluster size splits this mix (40 / 8 is below the HDM halo),
        # so the tuner picks the grid form or the grouped cluster form
        assert b.cluster() in (0, -1)
        assert threads in (128, 256, 512, 1024) and grid > 0
        assert (threads, grid) == b.launch()
        after = b.density()
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        b.step(10)
        b.sync()


def test_batch_barrier_timeout_is_reported_without_hanging():
    pairs = [instance(*m[:5], force=m[5], grad=m[6], prec="f32") for m in MIX[:3]]
    rho0 = [inputs.slab(op.nx, op.ny, *oracle.maxwell(op)[:2]) for _, op in pairs]
    with lbm.Batch([gp for gp, _ in pairs]) as b:
        b.init_density(rho0)
        b.debug_skip_barrier(0, 0.2)   # block 0 never arrives: the others give up after 0.2 s
        b.step(3)
        with pytest.raises(lbm.LBMError) as ei:
            b.sync()
        assert ei.value.status == lbm.E_TIMEOUT
        b.debug_skip_barrier(-1, 2.0)
        b.init_density(rho0)
        b.step(3)
        b.sync()


def test_full_sweep_coexistence_against_maxwell():
    # the 64-lattice sweep as the benchmark runs it (Nx uniform in [256, 2048],
    # EOS drawn from {VdW, CS, PR, RK}, T/Tc 0.5-0.95, tau in [0.8, 1.2], FP32,
    # SC + HDM, the tuned launch) for 20000 steps: HDM coexistence densities
    # against the Maxwell construction (Sec. 5.2), liquid within 2 %, vapour
    # within 10 %.  The PR lattices below T/Tc 0.6 (density ratio above 800)
    # relax their vapour phase more slowly than 20000 steps allow: for them
    # the test asserts instead that the batch follows the FP64 oracle's run of
    # the same lattice, so what remains is the model's, not the kernel's.
    table = inputs.sweep_instances(64)
    params, rho0, ref = [], [], []
    for d in table:
        gp = lbm.Params(nx=d["nx"], ny=d["ny"], eos=d["eos"], a=d["a"], b=d["b"], omega=d["omega"], Tr=d["Tr"],
                        k=d["k"], tau=d["tau"], force="sc", grad="hdm", prec="f32")
        g, l = lbm.maxwell(gp)
        params.append(gp)
        rho0.append(inputs.slab(d["nx"], d["ny"], g, l))
        ref.append((g, l))
    assert any(p.nx % 8 for p in params)   # widths the cluster form splits unevenly
    with lbm.Batch(params) as b:
        b.init_density(rho0)
        b.tune(trial_steps=20)
        b.init_density(rho0)
        b.step(20000)
        rho = b.density()
    slow = []
    for gp, r, (g, l), d in zip(params, rho, ref, table):
        liq, gas = bulk_slab(r)
        print(f"{gp.eos} T/Tc {gp.Tr:.3f} nx {gp.nx}: rho_l {liq / l - 1:+.2%} rho_g {gas / g - 1:+.2%}")
        if gp.eos == "pr" and gp.Tr < 0.6:
            slow.append((gp, r, d))
            continue
        assert abs(liq / l - 1) < 0.02, (gp.eos, gp.Tr, liq, l)
        assert abs(gas / g - 1) < 0.10, (gp.eos, gp.Tr, gas, g)
    oracle.set_threads(oracle.max_threads())
    for gp, r, d in slow:
        op = oracle.params_at(gp.nx, 8, "pr", d["a"], d["b"], gp.Tr, omega=d["omega"], k=d["k"], tau=gp.tau)
        ro = oracle.run(op, oracle.init(op, inputs.slab(gp.nx, 8, *oracle.maxwell(op)[:2])), 20000).sum(0)
        liq, gas = bulk_slab(r)
        liq_o, gas_o = bulk_slab(ro)
        assert abs(liq / liq_o - 1) < 1e-3 and abs(gas / gas_o - 1) < 1e-2, (gp.Tr, liq, liq_o, gas, gas_o)


def bulk_slab(r):
    prof = r.mean(0)
    nx = prof.size
    liq = prof[nx // 2 - nx // 16: nx // 2 + nx // 16 + 1].mean()
    gas = np.r_[prof[: nx // 16 + 1], prof[-nx // 16:]].mean()
    return liq, gas


def test_batch_sweep_coexistence_close_to_maxwell():
    # a reduced sweep (8 instances, 8000 steps, past the interface transient that
    # the oracle shows on the same lattices): HDM coexistence vs Maxwell (Sec. 5.2)
    table = inputs.sweep_instances(8, tr_lo=0.7, tr_hi=0.9)
    params, rho0, ref = [], [], []
    for d in table:
        nx = max(256, min(d["nx"], 512))
        gp = lbm.Params(nx=nx, ny=8, eos=d["eos"], a=d["a"], b=d["b"], omega=d["omega"], Tr=d["Tr"], k=d["k"],
                        tau=d["tau"], force="sc", grad="hdm", prec="f32")
        g, l = lbm.maxwell(gp)
        params.append(gp)
        rho0.append(inputs.slab(nx, 8, g, l))
        ref.append((g, l))
    with lbm.Batch(params) as b:
        b.init_density(rho0)
        b.step(8000)
        rho = b.density()
    for gp, r, (g, l) in zip(params, rho, ref):
        prof = r.mean(0)
        nx = gp.nx
        liq = prof[nx // 2 - nx // 16: nx // 2 + nx // 16 + 1].mean()
        gas = np.r_[prof[: nx // 16 + 1], prof[-nx // 16:]].mean()
        assert abs(liq / l - 1) < 0.02, (gp.eos, gp.Tr, liq, l)
        assert abs(gas / g - 1) < 0.10, (gp.eos, gp.Tr, gas, g)
