"""Host-side pieces of the benchmark that need no GPU: the oracle's CPU
baseline samples (all host threads, then one thread, then all threads again:
a one-thread sample must not leave the oracle single-threaded) and the
comment-insensitive digest that keys the recorded DRAM traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_samples_restore_the_thread_count():
    m_all, used_all, _ = bench.oracle_sample(64, 1)
    m_one, used_one, _ = bench.oracle_sample(64, 1, threads=1)
    m_again, used_again, _ = bench.oracle_sample(64, 1)
    assert used_one == 1
    assert used_all == used_again >= 1
    assert m_all > 0 and m_one > 0 and m_again > 0


def test_source_digest_ignores_comments_only():
    src = "int a; // x\n/* block\n comment */ int b = 1;  \n"
    same = "int a;\nint b = 1; // other words\n"
    assert bench.strip_comments(src) == bench.strip_comments(same)
    assert bench.strip_comments("int a = 1;") != bench.strip_comments("int a = 2;")
    # string literals keep their comment-like contents
    assert "//" in bench.strip_comments('const char *s = "a // b";')


def test_launch_time_uses_the_timed_region_only_for_a_single_kernel():
    # one kernel, one launch per step: the region's time over the launches
    t = {"steps": 100, "launches": 100, "kernels": {"fused_step": {"ms": 23.0, "count": 100}}}
    k, launch_ms, iso, n, only = bench.launch_time(t, region_ms=22.0 * 2, steps=200)
    assert (k, n, only) == ("fused_step", 200, True)
    assert abs(launch_ms - 0.22) < 1e-12 and abs(iso - 0.23) < 1e-12
    # two kernels per step (the two-pass path): the serialised per-launch time of the dominant one
    t = {"steps": 10, "launches": 20,
         "kernels": {"potential": {"ms": 1.0, "count": 10}, "collide": {"ms": 5.0, "count": 10}}}
    k, launch_ms, iso, n, only = bench.launch_time(t, region_ms=70.0, steps=10)
    assert (k, n, only) == ("collide", 20, False)
    assert launch_ms == iso == 0.5
