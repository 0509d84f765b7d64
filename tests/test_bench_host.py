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
